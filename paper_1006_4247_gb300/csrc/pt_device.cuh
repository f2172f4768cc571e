// pt_device.cuh -- device building blocks of the engine: counter-based random
// numbers, checkerboard geometry, and the single-site moves of Hasenbusch &
// Schaefer (arXiv:1006.4247) in float and double.
#pragma once
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "pt_types.h"

namespace ptk {

// ---------------------------------------------------------------------------
// Fast division (see FastDiv).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
    return f.m == 0u ? n : (__umulhi(n, f.m) >> f.s);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// multiplications with a Weyl-sequence key schedule.  Counter layout:
// (c0, c1, step_lo, purpose << 24 | step_hi); key (seed_lo, seed_hi ^ sample).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint4 rng_words(uint64_t seed, uint32_t sample, uint32_t c0,
                                           uint32_t c1, uint64_t step, uint32_t purpose) {
    const uint2 k = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32) ^ sample);
    const uint4 c = make_uint4(c0, c1, (uint32_t)step,
                               (purpose << 24) | ((uint32_t)(step >> 32) & 0xFFFFFFu));
    return philox4x32_10(c, k);
}

// u in [0,1) with 53 bits from two words.
__device__ __forceinline__ double u53(uint32_t w0, uint32_t w1) {
    return ((double)(w0 >> 5) * 67108864.0 + (double)(w1 >> 6)) * 0x1p-53;
}

// ---------------------------------------------------------------------------
// Checkerboard geometry of one sample.
// ---------------------------------------------------------------------------
struct Site {
    int h;              // index within the colour
    int ih, j, k, i;    // coordinates
    int x;              // natural site index i + L (j + L k)
    int xp, xm;         // h of the +x / -x neighbours (other colour)
    int yp, ym, zp, zm; // h of the +-y, +-z neighbours (other colour)
};

__device__ __forceinline__ Site site_of(const SampleDesc& sd, int color, int h) {
    Site st;
    st.h = h;
    const uint32_t row = fdiv((uint32_t)h, sd.div_hL);
    st.ih = h - (int)row * sd.hL;
    const uint32_t kk = fdiv(row, sd.div_L);
    st.k = (int)kk;
    st.j = (int)row - st.k * sd.L;
    const int p = (st.j + st.k + color) & 1;
    st.i = 2 * st.ih + p;
    st.x = st.i + sd.L * ((int)row);
    const int hL = sd.hL, L = sd.L;
    const int rowbase = (int)row * hL;
    // x neighbours: same row of the other colour
    int ixp = p ? st.ih + 1 : st.ih;
    if (ixp == hL) ixp = 0;
    int ixm = p ? st.ih : st.ih - 1;
    if (ixm < 0) ixm = hL - 1;
    st.xp = rowbase + ixp;
    st.xm = rowbase + ixm;
    const int jp = (st.j + 1 == L) ? 0 : st.j + 1;
    const int jm = (st.j == 0) ? L - 1 : st.j - 1;
    const int kp = (st.k + 1 == L) ? 0 : st.k + 1;
    const int km = (st.k == 0) ? L - 1 : st.k - 1;
    st.yp = st.ih + hL * (jp + L * st.k);
    st.ym = st.ih + hL * (jm + L * st.k);
    st.zp = st.ih + hL * (st.j + L * kp);
    st.zm = st.ih + hL * (st.j + L * km);
    return st;
}

// ---------------------------------------------------------------------------
// Precision-dependent math.
// ---------------------------------------------------------------------------
template <typename T> struct M;
template <> struct M<float> {
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
    static __device__ __forceinline__ float log_(float x) { return logf(x); }
    static __device__ __forceinline__ float log1p_(float x) { return log1pf(x); }
    static __device__ __forceinline__ float exp_(float x) { return expf(x); }
    static __device__ __forceinline__ float expm1_(float x) { return expm1f(x); }
    static __device__ __forceinline__ void sincos_(float x, float* s, float* c) { sincosf(x, s, c); }
    static __device__ __forceinline__ float sin_(float x) { return sinf(x); }
    static __device__ __forceinline__ float cos_(float x) { return cosf(x); }
    static __device__ __forceinline__ float atan2_(float y, float x) { return atan2f(y, x); }
    static __device__ __forceinline__ float copysign_(float a, float b) { return copysignf(a, b); }
    static constexpr float tinyR = 1e-30f;
    static constexpr int newton_max = 30;
    // heating step: after a Newton step of size d the root is within
    // e / (2 (1 - e)) d^2 (f'' = e sin, f' >= 1 - e), so stopping at
    // |d| < 1e-4 leaves < 5e-8 rad even at e = 0.9 (the float ulp of an angle
    // ~1 is 6e-8), one iteration earlier than |d| < 2e-7
    static constexpr float newton_tol = 1e-4f;
    static constexpr float pi = CUDART_PI_F;
};
template <> struct M<double> {
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ double rsqrt_(double x) { return 1.0 / sqrt(x); }
    static __device__ __forceinline__ double log_(double x) { return log(x); }
    static __device__ __forceinline__ double log1p_(double x) { return log1p(x); }
    static __device__ __forceinline__ double exp_(double x) { return exp(x); }
    static __device__ __forceinline__ double expm1_(double x) { return expm1(x); }
    static __device__ __forceinline__ void sincos_(double x, double* s, double* c) { sincos(x, s, c); }
    static __device__ __forceinline__ double sin_(double x) { return sin(x); }
    static __device__ __forceinline__ double cos_(double x) { return cos(x); }
    static __device__ __forceinline__ double atan2_(double y, double x) { return atan2(y, x); }
    static __device__ __forceinline__ double copysign_(double a, double b) { return copysign(a, b); }
    static constexpr double tinyR = 1e-280;
    static constexpr int newton_max = 50;
    static constexpr double newton_tol = 1e-15;
    static constexpr double pi = CUDART_PI;
};

// Quotients, square roots and the azimuth of the heat bath, cooling and
// heating steps.  Float takes the hardware forms: the reciprocal quotient
// (2 ulp; every divisor is O(1), an angle, or |S| of a site), the reciprocal
// square root (2 ulp), and sin/cos of pi x, whose argument reduction is exact
// (the azimuth is 2 pi u with u on a 2^-24 grid, so 2u is exact).  Double
// divides, takes the square root and the sine and cosine of 2 pi u.
template <typename T> struct MX;
template <> struct MX<float> {
    static __device__ __forceinline__ float div_(float a, float b) { return __fdividef(a, b); }
    // |S| and 1 / |S| from |S|^2 > 0
    static __device__ __forceinline__ void len_inv_(float x, float& n, float& inv) {
        inv = rsqrtf(x);
        n = x * inv;
    }
    // sqrt(x), x >= 0
    static __device__ __forceinline__ float sqrt0_(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }
    // sin and cos of 2 pi u
    static __device__ __forceinline__ void sincos_turn_(float u, float* s, float* c) { sincospif(2.0f * u, s, c); }
};
template <> struct MX<double> {
    static __device__ __forceinline__ double div_(double a, double b) { return a / b; }
    static __device__ __forceinline__ void len_inv_(double x, double& n, double& inv) {
        n = sqrt(x);
        inv = 1.0 / n;
    }
    static __device__ __forceinline__ double sqrt0_(double x) { return sqrt(x); }
    static __device__ __forceinline__ void sincos_turn_(double u, double* s, double* c) {
        sincos(2.0 * CUDART_PI * u, s, c);
    }
};

template <typename T> struct V3 { T x, y, z; };

template <typename T>
__device__ __forceinline__ T dot(const V3<T>& a, const V3<T>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// s <- s / |s|.  Every caller rotates, reflects or builds a unit vector from
// unit vectors (spins enter the engine normalised: pt_set_spins normalises,
// initial spins are unit), so |s|^2 = 1 + d with d a few rounding errors.  The
// factor is then the first Newton step for x^(-1/2) at x = 1, 1 - d/2 (one
// FMA), whose error 3d^2/8 is below the result's rounding.  Float always takes
// it: it replaces the hardware reciprocal square root, whose error has a sign
// bias (renormalising with it left |s|^2 - 1 at -8e-8 on average, i.e. spins
// a little short and energies scaled by 1 - 8e-8), while one rounded FMA
// rounds both ways.  Double guards |d| < 1e-8 and otherwise divides by the
// square root; the Newton form saves a square root and a division on GB300's
// slow FP64 pipe.
template <typename T>
__device__ __forceinline__ void renorm(V3<T>& s) {
    const T ss = dot(s, s);
    T inv;
    if (sizeof(T) == 4 || fabs(ss - (T)1) < (T)1e-8) inv = (T)1.5 - (T)0.5 * ss;
    else inv = M<T>::rsqrt_(ss);
    s.x *= inv; s.y *= inv; s.z *= inv;
}

// Spin of colour array `arr` (base of [comp][half]) at h.
template <typename T>
__device__ __forceinline__ V3<T> ld3(const T* __restrict__ arr, int half, int h) {
    V3<T> v;
    v.x = arr[h];
    v.y = arr[half + h];
    v.z = arr[2 * half + h];
    return v;
}
template <typename T>
__device__ __forceinline__ void st3(T* __restrict__ arr, int half, int h, const V3<T>& v) {
    arr[h] = v.x;
    arr[half + h] = v.y;
    arr[2 * half + h] = v.z;
}

// Neighbour field S_x = sum_y J_xy s_y (Eq. bigS).  `other` is the other
// colour's [comp][half] array, Jown / Joth the colour-split forward couplings
// ([mu][half]) of the site's colour and of the other colour.
template <typename T>
__device__ __forceinline__ V3<T> local_field(const Site& st, int half, const T* __restrict__ other,
                                             const float* __restrict__ Jown,
                                             const float* __restrict__ Joth) {
    const T jxp = (T)__ldg(Jown + st.h), jyp = (T)__ldg(Jown + half + st.h),
            jzp = (T)__ldg(Jown + 2 * half + st.h);
    const T jxm = (T)__ldg(Joth + st.xm), jym = (T)__ldg(Joth + half + st.ym),
            jzm = (T)__ldg(Joth + 2 * half + st.zm);
    V3<T> S;
    S.x = jxp * other[st.xp] + jxm * other[st.xm] + jyp * other[st.yp] + jym * other[st.ym] +
          jzp * other[st.zp] + jzm * other[st.zm];
    const T* oy = other + half;
    S.y = jxp * oy[st.xp] + jxm * oy[st.xm] + jyp * oy[st.yp] + jym * oy[st.ym] +
          jzp * oy[st.zp] + jzm * oy[st.zm];
    const T* oz = other + 2 * half;
    S.z = jxp * oz[st.xp] + jxm * oz[st.xm] + jyp * oz[st.yp] + jym * oz[st.ym] +
          jzp * oz[st.zp] + jzm * oz[st.zm];
    return S;
}

// ---------------------------------------------------------------------------
// Heat bath (section III.C): cos(theta) along n = S/|S| from the inverse of
// its conditional distribution, t = 1 - cos(theta) =
// -ln(1 - q (1 - e^{-2R})) / R with R = beta |S| and q = 1 - r; the logarithm's
// argument equals r + q e^{-2R}.  Azimuth phi in the basis of Duff et al.
// (JCGT 2017) around n.  r and phi come from the two words w0, w1.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ V3<T> hb_site(T beta, const V3<T>& S, uint32_t w0, uint32_t w1) {
    const T nS2 = dot(S, S);
    T nS;
    V3<T> n;
    if (nS2 > (T)0) {
        T inv;
        MX<T>::len_inv_(nS2, nS, inv);
        n.x = S.x * inv; n.y = S.y * inv; n.z = S.z * inv;
    } else {
        nS = (T)0;
        n.x = (T)0; n.y = (T)0; n.z = (T)1;
    }
    const T R = beta * nS;
    const T q = (T)(0xFFFFFFu - (w0 >> 8)) * (T)0x1p-24;
    T t;
    if (R < M<T>::tinyR) {
        t = (T)2 * q;
    } else {
        const T a = -M<T>::expm1_((T)-2 * R);
        const T qa = q * a;
        if (qa <= (T)0.5)
            t = MX<T>::div_(-M<T>::log1p_(-qa), R);
        else
            t = MX<T>::div_(-M<T>::log_(((T)1 - q) + q * M<T>::exp_((T)-2 * R)), R);
    }
    t = t < (T)0 ? (T)0 : (t > (T)2 ? (T)2 : t);
    const T c = (T)1 - t;
    const T st = MX<T>::sqrt0_(t * ((T)2 - t));
    T sp, cp;
    MX<T>::sincos_turn_((T)(w1 >> 8) * (T)0x1p-24, &sp, &cp);
    const T sgn = M<T>::copysign_((T)1, n.z);
    const T a = MX<T>::div_((T)-1, sgn + n.z);  // |sgn + n.z| >= 1
    const T b = n.x * n.y * a;
    const V3<T> e1 = {(T)1 + sgn * n.x * n.x * a, sgn * b, -sgn * n.x};
    const V3<T> e2 = {b, sgn + n.y * n.y * a, -n.y};
    V3<T> s;
    s.x = c * n.x + st * (sp * e1.x + cp * e2.x);
    s.y = c * n.y + st * (sp * e1.y + cp * e2.y);
    s.z = c * n.z + st * (sp * e1.z + cp * e2.z);
    renorm(s);
    return s;
}

// Overrelaxation (section III.C): reflection of s about S; S = 0 keeps s.
// In float the quotient uses the hardware reciprocal (2 ulp).
__device__ __forceinline__ float or_quot(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double or_quot(double a, double b) { return a / b; }

template <typename T>
__device__ __forceinline__ void or_site(const V3<T>& S, V3<T>& s) {
    const T SS = dot(S, S);
    if (SS > (T)0) {
        const T f = or_quot((T)2 * dot(s, S), SS);
        s.x = f * S.x - s.x;
        s.y = f * S.y - s.y;
        s.z = f * S.z - s.z;
        renorm(s);
    }
}

// ln(sinh R / R) = ln of I(beta S) / (4 pi) (Eq. HI); ln[2 sinh R] = R +
// ln[1 - e^{-2R}] (appendix A).
template <typename T>
__device__ __forceinline__ T ln_sinhc(T R) {
    if (R == (T)0) return (T)0;
    if (R < (T)0.5) {
        // ln(sinh R / R) = ln(-expm1(-2R) / (2R)) + R, accurate for small R
        return M<T>::log_(-M<T>::expm1_((T)-2 * R) / ((T)2 * R)) + R;
    }
    return R + M<T>::log1p_(-M<T>::exp_((T)-2 * R)) - M<T>::log_((T)2 * R);
}

// Rotation angle functions of the cooling and heating steps: cos(a) - 1 and
// sin(a) / a.  The angle obeys 0 <= a <= eps |S| < 1 (the invertibility
// bound of section III.B), so in float both are taken from their Taylor
// series, truncated after the a^10 term (remainder below a^12 / 12! and
// a^12 / 13!, i.e. under 2.1e-9 relative on [0, 1)): they keep full relative
// accuracy at the small angles of the method, where cos(a) - 1 would lose
// every digit to cancellation and the hardware sine has an absolute, not a
// relative, error.  Double uses the library functions.
template <typename T> struct Rot;
template <> struct Rot<float> {
    static __device__ __forceinline__ void cs(float a, float& cm1, float& sc) { cs2(a * a, cm1, sc); }
    // from a^2 (both series are even): the cooling step needs no square root
    static __device__ __forceinline__ void cs2(float a2, float& cm1, float& sc) {
        // cos a - 1 = -a^2/2! + a^4/4! - a^6/6! + a^8/8! - a^10/10!
        float c = -2.7557319e-7f;
        c = fmaf(c, a2, 2.4801587e-5f);
        c = fmaf(c, a2, -1.3888889e-3f);
        c = fmaf(c, a2, 4.1666668e-2f);
        c = fmaf(c, a2, -0.5f);
        cm1 = c * a2;
        // sin a / a = 1 - a^2/3! + a^4/5! - a^6/7! + a^8/9! - a^10/11!
        float t = -2.5052108e-8f;
        t = fmaf(t, a2, 2.7557319e-6f);
        t = fmaf(t, a2, -1.9841270e-4f);
        t = fmaf(t, a2, 8.3333333e-3f);
        t = fmaf(t, a2, -0.16666667f);
        sc = fmaf(t, a2, 1.0f);
    }
};
template <> struct Rot<double> {
    static __device__ __forceinline__ void cs(double a, double& cm1, double& sc) {
        cm1 = cos(a) - 1.0;
        sc = a == 0.0 ? 1.0 : sin(a) / a;
    }
    static __device__ __forceinline__ void cs2(double a2, double& cm1, double& sc) { cs(sqrt(a2), cm1, sc); }
};

// log(1 + x) in float for the small arguments of ln_jac: with
// z = x / (2 + x), log(1 + x) = 2 atanh z = 2 (z + z^3/3 + ... + z^9/9), the
// series cut after z^9 (relative remainder below z^10 / 11: 1e-8 at
// |x| = 0.5, z = 0.2, and far less at the method's |x| ~ 0.1); the quotient
// is the hardware one (2 ulp, so a few 1e-7 relative, i.e. ~1e-8 absolute).  Larger |x| (not met while
// eps |S| is well below 1) take the library log1p.
__device__ __forceinline__ float log1p_small(float x) {
    if (fabsf(x) > 0.5f) return log1pf(x);
    const float z = __fdividef(x, 2.0f + x), z2 = z * z;
    float t = 1.0f / 9.0f;
    t = fmaf(t, z2, 1.0f / 7.0f);
    t = fmaf(t, z2, 0.2f);
    t = fmaf(t, z2, 1.0f / 3.0f);
    t = fmaf(t, z2, 1.0f);
    return 2.0f * z * t;
}
__device__ __forceinline__ double log1p_small(double x) { return log1p(x); }

// ln det J_f of one elementary step, ln[(1 - q)(cos a - q sin(a)/a)], with
// q = eps (S.s) (cooling) or e cos(theta) (heating, at the pre-image).  In
// float the product is written as 1 + x with x = d - q - q d,
// d = (cos a - 1) - q sin(a)/a, and the logarithm taken as log1p(x): every
// quantity is formed at the size it has (x is small), so the per-site value
// is accurate to a few units in the last place of x instead of carrying the
// absolute error of a logarithm near 1, which summed over N sites would bias
// ln det J_C by O(N 1e-7).  Double keeps ln|j| of the product (the oracle's
// form).
template <typename T>
__device__ __forceinline__ T ln_jac(T q, T ca, T cm1, T sc) {
    if (sizeof(T) == 4) {
        const T d = cm1 - q * sc;
        return log1p_small(d - q - q * d);
    }
    return M<T>::log_(fabs(((T)1 - q) * (ca - q * sc)));
}

// Cooling step (section III.B): rotate s towards S by alpha = eps |p|,
// p = S - (S.s) s; returns ln det J_f = ln[(1 - eps S.s)(cos a - eps S.s sinc a)].
template <typename T>
__device__ __forceinline__ T cool_site(T eps, const V3<T>& S, V3<T>& s) {
    const T sS = dot(s, S);
    const V3<T> p = {S.x - sS * s.x, S.y - sS * s.y, S.z - sS * s.z};
    // alpha = eps |p| enters only through its square
    T cm1, sc;
    Rot<T>::cs2(eps * eps * dot(p, p), cm1, sc);
    const T ca = (T)1 + cm1;
    const T f = eps * sc;
    s.x = s.x * ca + p.x * f;
    s.y = s.y * ca + p.y * f;
    s.z = s.z * ca + p.z * f;
    renorm(s);
    return ln_jac<T>(eps * sS, ca, cm1, sc);
}

// Heating step = inverse cooling step: theta' (angle between s' and S) given,
// find theta with theta - e sin(theta) = theta', e = eps |S| < 1, and rotate
// s' away from S by alpha = theta - theta'.  The unknown is taken to be alpha
// itself: alpha = e sin(theta' + alpha), solved by Newton's method starting
// at its first step from 0, e sin(theta') / (1 - e cos(theta')), with
// cos(theta') = s'.S/|S| and sin(theta') = |p|/|S| read off the geometry, so
// no angle is ever formed.  At the solution
// alpha = e sin(theta), hence the Jacobian factors and the rotation reuse
// sin(alpha), cos(alpha).  Returns ln det J_f at the pre-image,
// ln[(1 - e cos(theta))(cos(alpha) - e cos(theta) sin(alpha)/alpha)].
template <typename T>
__device__ __forceinline__ T heat_site(T eps, const V3<T>& S, V3<T>& s) {
    const T nS = M<T>::sqrt_(dot(S, S));
    const T sS = dot(s, S);
    const V3<T> p = {S.x - sS * s.x, S.y - sS * s.y, S.z - sS * s.z};
    const T pn = M<T>::sqrt_(dot(p, p));
    const T e = eps * nS;
    const T inv = nS > (T)0 ? MX<T>::div_((T)1, nS) : (T)0;
    const T cp = nS > (T)0 ? sS * inv : (T)1;  // cos(theta')
    const T sp = pn * inv;                     // sin(theta')
    // start from the first Newton step from alpha = 0: e sin(theta') / (1 - e cos(theta'))
    T alpha = MX<T>::div_(e * sp, (T)1 - e * cp), cm1, sc;
    Rot<T>::cs(alpha, cm1, sc);
    T sa = alpha * sc, ca = (T)1 + cm1;
    for (int it = 0; it < M<T>::newton_max; ++it) {
        // f = alpha - e sin(theta' + alpha), f' = 1 - e cos(theta' + alpha)
        const T sth = sp * ca + cp * sa, cth = cp * ca - sp * sa;
        const T d = MX<T>::div_(alpha - e * sth, (T)1 - e * cth);  // only the path to the root
        alpha -= d;
        Rot<T>::cs(alpha, cm1, sc);
        sa = alpha * sc;
        ca = (T)1 + cm1;
        if (fabs(d) < M<T>::newton_tol) break;
    }
    if (pn > (T)0) {
        const T f = MX<T>::div_(sa, pn);
        s.x = s.x * ca - p.x * f;
        s.y = s.y * ca - p.y * f;
        s.z = s.z * ca - p.z * f;
        renorm(s);
    }
    const T cth = cp * ca - sp * sa;  // cos(theta)
    return ln_jac<T>(e * cth, ca, cm1, sc);
}

// ---------------------------------------------------------------------------
// Vector loads / stores of V consecutive elements (V * sizeof(T) = 4, 8, 16).
// ---------------------------------------------------------------------------
template <typename T, int V> struct VecT;
template <> struct VecT<float, 1> { using t = float; };
template <> struct VecT<float, 2> { using t = float2; };
template <> struct VecT<float, 4> { using t = float4; };
template <> struct VecT<double, 1> { using t = double; };
template <> struct VecT<double, 2> { using t = double2; };

template <typename T, int V>
__device__ __forceinline__ void ldv(const T* __restrict__ p, T (&o)[V]) {
    const typename VecT<T, V>::t v = *reinterpret_cast<const typename VecT<T, V>::t*>(p);
    const T* q = reinterpret_cast<const T*>(&v);
#pragma unroll
    for (int i = 0; i < V; ++i) o[i] = q[i];
}
template <typename T, int V>
__device__ __forceinline__ void ldv_nc(const T* __restrict__ p, T (&o)[V]) {
    const typename VecT<T, V>::t v = __ldg(reinterpret_cast<const typename VecT<T, V>::t*>(p));
    const T* q = reinterpret_cast<const T*>(&v);
#pragma unroll
    for (int i = 0; i < V; ++i) o[i] = q[i];
}
template <typename T, int V>
__device__ __forceinline__ void stv(T* __restrict__ p, const T (&o)[V]) {
    typename VecT<T, V>::t v;
    T* q = reinterpret_cast<T*>(&v);
#pragma unroll
    for (int i = 0; i < V; ++i) q[i] = o[i];
    *reinterpret_cast<typename VecT<T, V>::t*>(p) = v;
}

// ---------------------------------------------------------------------------
// Neighbour field of V consecutive sites h0 .. h0+V-1 of one row (Eq. bigS),
// direction by direction: for each of the six directions the coupling vector
// and the three component vectors of the neighbours are loaded, accumulated
// into S and dropped, so few registers stay live.  `oth` is the other
// colour's [comp][half] array, Jown / Joth the forward couplings of the two
// colours; p is the row's checkerboard offset, xs the index of the +-x
// neighbour that wraps around the row, hy*/hz* the rows' first indices.
// ---------------------------------------------------------------------------
// J_SHARED: the couplings live in shared memory (plain loads); otherwise in
// global memory, read through the read-only data cache.
template <bool J_SHARED, int V>
__device__ __forceinline__ void ldj(const float* __restrict__ p, float (&o)[V]) {
    if (J_SHARED) ldv<float, V>(p, o);
    else ldv_nc<float, V>(p, o);
}

// XSHFL: the row's vectors lie in consecutive lanes of the warp (all lanes
// active), so the element just outside the vector -- the other colour's
// first element of the next vector (p = 1) or last of the previous one
// (p = 0), wrapping around the row -- is taken from lane `xs` by a shuffle
// instead of a load (p is the same for every vector of a row).
template <typename T, int V, bool J_SHARED = false, bool XSHFL = false>
__device__ __forceinline__ void nbr_field(const T* __restrict__ oth, const float* __restrict__ Jown,
                                          const float* __restrict__ Joth, int half, int h0, int xs,
                                          int hyp, int hym, int hzp, int hzm, int p, T (&S)[3][V]) {
    {   // +-x: the same row of the other colour, shifted by one (plus xs)
        float jp[V], jm[V];
        ldj<J_SHARED, V>(Jown + h0, jp);
        {
            float jx[V];
            ldj<J_SHARED, V>(Joth + h0, jx);
            const float jxs = XSHFL ? __shfl_sync(0xFFFFFFFFu, jx[V - 1], xs)
                                    : (J_SHARED ? Joth[xs] : __ldg(Joth + xs));
#pragma unroll
            for (int v = 0; v < V; ++v) jm[v] = p ? jx[v] : (v == 0 ? jxs : jx[v - 1]);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T* o = oth + c * half;
            T O[V];
            ldv<T, V>(o + h0, O);
            const T os = XSHFL ? __shfl_sync(0xFFFFFFFFu, p ? O[0] : O[V - 1], xs) : o[xs];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const T xp = p ? (v == V - 1 ? os : O[v + 1]) : O[v];
                const T xm = p ? O[v] : (v == 0 ? os : O[v - 1]);
                S[c][v] = (T)jp[v] * xp + (T)jm[v] * xm;
            }
        }
    }
    const float* jsrc[4] = {Jown + half + h0, Joth + half + hym, Jown + 2 * half + h0, Joth + 2 * half + hzm};
    const int nrow[4] = {hyp, hym, hzp, hzm};
#pragma unroll
    for (int dir = 0; dir < 4; ++dir) {
        float jd[V];
        ldj<J_SHARED, V>(jsrc[dir], jd);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            T n[V];
            ldv<T, V>(oth + c * half + nrow[dir], n);
#pragma unroll
            for (int v = 0; v < V; ++v) S[c][v] += (T)jd[v] * n[v];
        }
    }
}

// Row indices of the V-site vector at h0 of colour `color` (the layout of the
// half sweeps): wrapped x neighbour, y and z neighbour rows, checkerboard
// offset p and the row number.
struct VRow {
    int xs, hyp, hym, hzp, hzm, p, row, ih0;
};

template <int V>
__device__ __forceinline__ VRow vrow(const SampleDesc& sd, int color, int h0) {
    const int hL = sd.hL, L = sd.L;
    VRow q;
    q.row = (int)fdiv((uint32_t)h0, sd.div_hL);
    q.ih0 = h0 - q.row * hL;
    const int k = (int)fdiv((uint32_t)q.row, sd.div_L);
    const int j = q.row - k * L;
    q.p = (j + k + color) & 1;
    const int rb = q.row * hL;
    q.xs = q.p ? rb + ((q.ih0 + V == hL) ? 0 : q.ih0 + V) : rb + ((q.ih0 == 0) ? hL - 1 : q.ih0 - 1);
    const int jp = (j + 1 == L) ? 0 : j + 1, jm = (j == 0) ? L - 1 : j - 1;
    const int kp = (k + 1 == L) ? 0 : k + 1, km = (k == 0) ? L - 1 : k - 1;
    q.hyp = q.ih0 + hL * (jp + L * k);
    q.hym = q.ih0 + hL * (jm + L * k);
    q.hzp = q.ih0 + hL * (j + L * kp);
    q.hzm = q.ih0 + hL * (j + L * km);
    return q;
}

// x 2^32 rounded to the nearest integer (ties to even) as a 64-bit integer,
// for |x| < 2^31: the same value as the 64-bit conversion of x 2^32, built
// from 32-bit conversions (GB300 runs 64-bit conversions on its narrow FP64
// pipe).  The integer part t of x, the next 16 fraction bits u and the rest
// are each exact in float (truncation only drops bits of x); only the last
// piece is rounded, and the pieces above it are multiples of 2^16, so
// rounding it rounds the whole.
__device__ __forceinline__ long long fixed32(float x) {
    const float t = truncf(x);
    const float f = (x - t) * 65536.0f;
    const float u = truncf(f);
    const int c = __float2int_rn((f - u) * 65536.0f);
    return (long long)(int)t * 4294967296LL + (long long)(int)u * 65536LL + (long long)c;
}

// ---------------------------------------------------------------------------
// Deterministic block reduction of a double (blockDim.x multiple of 32,
// <= 1024).  All threads must call it; the result is valid in thread 0.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Sum of NV values over the CTA, for values that each thread accumulated in
// T over its few sites: the 32 lanes of a warp are added in T, the warp sums
// in double (so float work stays on the float pipes and at most 32 float
// terms meet before the sum is carried in double).  One pass, two barriers;
// results valid in warp 0.  sh must hold NV * 32 doubles.  The warp sums
// are stored in T and widened by warp 0 (one conversion per value and lane
// instead of one per warp and value); with few warps and many values the
// warp sums of value k are then added by lane k in warp order (nw dependent
// double adds on NV lanes), else by a shuffle tree per value (5 NV double
// adds): whichever issues fewer instructions to GB300's slow FP64 pipe.
template <typename T, int NV>
__device__ __forceinline__ void block_sum_multi(const T (&v)[NV], double (&out)[NV], double* sh) {
    static_assert(NV <= 32, "one lane per value");
    T* shT = reinterpret_cast<T*>(sh);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        T x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
        if (lane == 0) shT[k * 32 + wid] = x;
    }
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    if (wid == 0) {
        if (2 * nw < 6 * NV) {
            double r = 0.0;
            if (lane < NV)
                for (int w = 0; w < nw; ++w) r += (double)shT[lane * 32 + w];
#pragma unroll
            for (int k = 0; k < NV; ++k) out[k] = __shfl_sync(0xFFFFFFFFu, r, k);
        } else {
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                double r = (lane < nw) ? (double)shT[k * 32 + lane] : 0.0;
                out[k] = warp_sum(r);
            }
        }
    }
}

// Knuth's two-sum accumulation: s + c carries the running sum of the added
// values to about twice the working precision (for threads that add many
// site terms before the block reduction).
template <typename T>
__device__ __forceinline__ void acc_add(T& s, T& c, T x) {
    const T t = s + x;
    const T bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
}

// Sum of NV per-thread values over the CTA for the exchange kernels.  Their
// totals (energies of proposals, ln det J_C, decimation sums) enter ln A
// multiplied by beta, and partial sums reach 10^3..10^4, where a float
// shuffle tree would lose ~1e-4 per warp.  Float values are therefore turned
// into 64-bit fixed point once per thread (resolution 2^-32; |total| < 2^31
// by far) and added exactly: integer addition is associative, so the result
// is the exact sum of the per-thread values for any reduction order or
// cluster size, rounded once to double (exactly, while |total| < 2^21).  The
// conversion (fixed32) and the adds run on the integer and FP32 pipes, not
// GB300's narrow FP64 one.  Double values take block_sum_multi.  Results valid
// in warp 0; sh holds NV * 32 doubles.
template <typename T, int NV>
__device__ __forceinline__ void block_sum_exact(const T (&v)[NV], double (&out)[NV], double* sh) {
    if (sizeof(T) == 8) {
        block_sum_multi<T, NV>(v, out, sh);
        return;
    }
    static_assert(NV <= 32, "one slot row per value");
    long long* shI = reinterpret_cast<long long*>(sh);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        long long x = fixed32((float)v[k]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
        if (lane == 0) shI[k * 32 + wid] = x;
    }
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            long long r = (lane < nw) ? shI[k * 32 + lane] : 0ll;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xFFFFFFFFu, r, o);
            out[k] = (double)r * 0x1p-32;
        }
    }
}

__device__ __forceinline__ double block_sum(double v, double* sh /* >= 32 doubles */) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    double r = 0.0;
    if (wid == 0) {
        r = (lane < nw) ? sh[lane] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

}  // namespace ptk
