/*
 * pt_oracle.c -- plain, slow FP64 CPU oracle for parallel tempering of the
 * three-dimensional Heisenberg Edwards-Anderson spin glass, following
 * M. Hasenbusch and S. Schaefer, "Speeding up parallel tempering simulations"
 * (arXiv:1006.4247).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference that the CUDA engine is
 * checked against.  Only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header or table with the
 * CUDA engine; both sides implement the counter-based generator from its
 * published definition.
 *
 * Everything is double precision and written site by site in the order the
 * method states it.  No blocking, no fusion, no vectorisation.
 *
 * Conventions (identical on both sides, stated here in full):
 *   L even or odd (odd L only in typewriter order), N = L^3 sites,
 *   site x = i + L*(j + L*k), colour c(x) = (i+j+k) mod 2 (0 = "black").
 *   Bond (x, mu) joins x and x + e_mu (periodic) with coupling J[mu*N + x].
 *   Spins: s[3*x + a], a = 0,1,2 (natural order, unit vectors).
 *   A chain is (sample, copy); within a chain the configuration at inverse
 *   temperature index b (betas increasing with b) is stored at spins[b].
 *   "label[b]" is the identity of the configuration at index b (for round
 *   trips); "H[b]" its Hamiltonian.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11).
 *   key = (seed_lo32, seed_hi32 XOR sample)
 *   ctr = (c0, c1, step_lo32, (purpose << 24) | (step_hi32 & 0xFFFFFF))
 *   purpose 0: heat bath        c0 = site x, c1 = copy*NT + b
 *   purpose 1: exchange uniform c0 = pair index i, c1 = copy
 *   purpose 2: decimation re-insertion heat bath, c0 = x, c1 = copy*NT + b
 *   purpose 3: decimation first colour, c0 = 0, c1 = copy
 *   purpose 4: initial spins    c0 = x, c1 = copy*NT + b, step = 0
 * Conversions of the 32-bit words w0, w1:
 *   r   = ((w0 >> 8) + 1) * 2^-24 in (0,1];  q = 1 - r, exact
 *   phi = 2 pi * (w1 >> 8) * 2^-24 in [0, 2 pi)
 *   u53 = ((w0 >> 5) * 2^26 + (w1 >> 6)) * 2^-53 in [0, 1)
 *   initial spin: z = (w0 >> 8) * 2^-23 - 1,  phi as above.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from the published definition (SC'11, section 2 and       */
/* table 2): two 32x32->64 multiplications per round, Weyl key schedule.    */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                       uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k[2] = {key_in[0], key_in[1]};
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k[0];
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c[3] ^ k[1];
        uint32_t n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
        k[0] += W0; k[1] += W1;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

void orc_rng_words(uint64_t seed, uint32_t sample, uint32_t c0, uint32_t c1,
                   uint64_t step, uint32_t purpose, uint32_t out[4])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ sample};
    uint32_t ctr[4] = {c0, c1, (uint32_t)step,
                       (purpose << 24) | ((uint32_t)(step >> 32) & 0xFFFFFFu)};
    orc_philox4x32_10(ctr, key, out);
}

double orc_uniform_r(uint32_t w0) { return (double)((w0 >> 8) + 1u) * 0x1p-24; }
double orc_uniform_q(uint32_t w0) { return (double)(0xFFFFFFu - (w0 >> 8)) * 0x1p-24; }
double orc_uniform_phi(uint32_t w1) { return 2.0 * ORC_PI * ((double)(w1 >> 8) * 0x1p-24); }
double orc_uniform_u53(uint32_t w0, uint32_t w1)
{
    return ((double)(w0 >> 5) * 67108864.0 + (double)(w1 >> 6)) * 0x1p-53;
}

/* ------------------------------------------------------------------------ */
/* Lattice: neighbours on the periodic simple-cubic lattice (section I).    */
/* ------------------------------------------------------------------------ */
static int site_index(int L, int i, int j, int k)
{
    i = ((i % L) + L) % L; j = ((j % L) + L) % L; k = ((k % L) + L) % L;
    return i + L * (j + L * k);
}

int orc_color(int L, int x)
{
    int i = x % L, j = (x / L) % L, k = x / (L * L);
    return (i + j + k) & 1;
}

/* Neighbour field S_x = sum over the six nearest neighbours y of J_xy s_y
 * (Eq. bigS of section III.A).  Bond (x, mu) carries J[mu*N + x]; the bond
 * to x - e_mu carries J[mu*N + (x - e_mu)]. */
void orc_local_field(int L, const double *J, const double *s, int x, double S[3])
{
    int N = L * L * L;
    int i = x % L, j = (x / L) % L, k = x / (L * L);
    int fwd[3] = {site_index(L, i + 1, j, k), site_index(L, i, j + 1, k),
                  site_index(L, i, j, k + 1)};
    int bwd[3] = {site_index(L, i - 1, j, k), site_index(L, i, j - 1, k),
                  site_index(L, i, j, k - 1)};
    S[0] = S[1] = S[2] = 0.0;
    for (int mu = 0; mu < 3; ++mu) {
        double jf = J[mu * N + x];
        double jb = J[mu * N + bwd[mu]];
        for (int a = 0; a < 3; ++a)
            S[a] += jf * s[3 * fwd[mu] + a] + jb * s[3 * bwd[mu] + a];
    }
}

/* H = - sum over bonds <xy> of J_xy s_x . s_y  (section I, Eq. H). */
double orc_energy(int L, const double *J, const double *s)
{
    int N = L * L * L;
    double H = 0.0;
    for (int x = 0; x < N; ++x) {
        int i = x % L, j = (x / L) % L, k = x / (L * L);
        int fwd[3] = {site_index(L, i + 1, j, k), site_index(L, i, j + 1, k),
                      site_index(L, i, j, k + 1)};
        for (int mu = 0; mu < 3; ++mu) {
            int y = fwd[mu];
            double d = s[3 * x] * s[3 * y] + s[3 * x + 1] * s[3 * y + 1] +
                       s[3 * x + 2] * s[3 * y + 2];
            H -= J[mu * N + x] * d;
        }
    }
    return H;
}

/* Overlap q_{ab,x} = s1_{a,x} s2_{b,x} summed over x (section II, Eq. over):
 * Q[3a + b]; chi = (1/N) sum_ab Q_ab^2. */
double orc_overlap(int L, const double *s1, const double *s2, double Q[9])
{
    int N = L * L * L;
    for (int n = 0; n < 9; ++n) Q[n] = 0.0;
    for (int x = 0; x < N; ++x)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                Q[3 * a + b] += s1[3 * x + a] * s2[3 * x + b];
    double chi = 0.0;
    for (int n = 0; n < 9; ++n) chi += Q[n] * Q[n];
    return chi / (double)N;
}

static void renormalise(double v[3])
{
    double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= n; v[1] /= n; v[2] /= n;
}

/* ------------------------------------------------------------------------ */
/* Heat bath (section III.C).  The component of the new spin along S is     */
/* c = ln(z + (1/z - z) r) / (beta |S|), z = exp(-beta |S|).  Written as     */
/* t = 1 - c = -log1p(-(1 - r)(1 - exp(-2R))) / R, R = beta |S|, which is    */
/* the same number without the overflow of 1/z.  The two orthogonal parts    */
/* are sqrt(1 - c^2) (sin phi, cos phi) in an orthonormal basis (e1, e2)     */
/* perpendicular to n = S/|S|.  The basis is that of Duff et al., "Building  */
/* an Orthonormal Basis, Revisited" (JCGT 6(1), 2017).  S = 0 (or R = 0)     */
/* gives the uniform distribution with n = e_z.                              */
/* ------------------------------------------------------------------------ */
void orc_onb(const double n[3], double e1[3], double e2[3])
{
    double sgn = (n[2] >= 0.0) ? 1.0 : -1.0;
    if (n[2] == 0.0 && signbit(n[2])) sgn = -1.0;
    double a = -1.0 / (sgn + n[2]);
    double b = n[0] * n[1] * a;
    e1[0] = 1.0 + sgn * n[0] * n[0] * a;
    e1[1] = sgn * b;
    e1[2] = -sgn * n[0];
    e2[0] = b;
    e2[1] = sgn + n[1] * n[1] * a;
    e2[2] = -n[1];
}

/* t = 1 - cos(theta) = -ln(1 - q (1 - e^{-2R})) / R.  The argument of the
 * logarithm equals r + q e^{-2R} (r = 1 - q exactly); log1p is used while
 * q (1 - e^{-2R}) <= 1/2 and the direct sum otherwise, so that neither end of
 * the r range loses digits. */
double orc_hb_t(double R, double q)
{
    double t;
    if (R < 1e-280) {
        t = 2.0 * q;
    } else {
        double a = -expm1(-2.0 * R);
        double qa = q * a;
        if (qa <= 0.5)
            t = -log1p(-qa) / R;
        else
            t = -log((1.0 - q) + q * exp(-2.0 * R)) / R;
    }
    if (t < 0.0) t = 0.0;
    if (t > 2.0) t = 2.0;
    return t;
}

void orc_hb_update(double beta, const double S[3], uint32_t w0, uint32_t w1,
                   double out[3])
{
    double nS = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
    double n[3];
    if (nS > 0.0) { n[0] = S[0] / nS; n[1] = S[1] / nS; n[2] = S[2] / nS; }
    else { n[0] = 0.0; n[1] = 0.0; n[2] = 1.0; }
    double R = beta * nS;
    double q = orc_uniform_q(w0);
    double t = orc_hb_t(R, q);
    double c = 1.0 - t;
    double st = sqrt(t * (2.0 - t));
    double phi = orc_uniform_phi(w1);
    double e1[3], e2[3];
    orc_onb(n, e1, e2);
    double sp = sin(phi), cp = cos(phi);
    for (int a = 0; a < 3; ++a)
        out[a] = c * n[a] + st * (sp * e1[a] + cp * e2[a]);
    renormalise(out);
}

/* Overrelaxation (section III.C): s' = 2 (s.S)/S^2 S - s; unchanged if S = 0. */
void orc_or_update(const double S[3], double s[3])
{
    double SS = S[0] * S[0] + S[1] * S[1] + S[2] * S[2];
    if (SS == 0.0) return;
    double f = 2.0 * (s[0] * S[0] + s[1] * S[1] + s[2] * S[2]) / SS;
    for (int a = 0; a < 3; ++a) s[a] = f * S[a] - s[a];
    renormalise(s);
}

/* One heat-bath half sweep of colour `color` (checkerboard; same-colour
 * sites do not interact, section III.A), random numbers with `purpose`. */
void orc_hb_halfsweep(int L, const double *J, double *s, int color, double beta,
                      uint64_t seed, uint32_t sample, uint32_t rep_id,
                      uint64_t step, uint32_t purpose)
{
    int N = L * L * L;
    for (int x = 0; x < N; ++x) {
        if (orc_color(L, x) != color) continue;
        double S[3], out[3];
        uint32_t w[4];
        orc_local_field(L, J, s, x, S);
        orc_rng_words(seed, sample, (uint32_t)x, rep_id, step, purpose, w);
        orc_hb_update(beta, S, w[0], w[1], out);
        s[3 * x] = out[0]; s[3 * x + 1] = out[1]; s[3 * x + 2] = out[2];
    }
}

void orc_or_halfsweep(int L, const double *J, double *s, int color)
{
    int N = L * L * L;
    for (int x = 0; x < N; ++x) {
        if (orc_color(L, x) != color) continue;
        double S[3];
        orc_local_field(L, J, s, x, S);
        orc_or_update(S, &s[3 * x]);
    }
}

/* Typewriter order (section III.C): every site in turn, x = 0 .. N-1. */
void orc_hb_sweep_typewriter(int L, const double *J, double *s, double beta,
                             uint64_t seed, uint32_t sample, uint32_t rep_id,
                             uint64_t step)
{
    int N = L * L * L;
    for (int x = 0; x < N; ++x) {
        double S[3], out[3];
        uint32_t w[4];
        orc_local_field(L, J, s, x, S);
        orc_rng_words(seed, sample, (uint32_t)x, rep_id, step, 0u, w);
        orc_hb_update(beta, S, w[0], w[1], out);
        s[3 * x] = out[0]; s[3 * x + 1] = out[1]; s[3 * x + 2] = out[2];
    }
}

void orc_or_sweep_typewriter(int L, const double *J, double *s)
{
    int N = L * L * L;
    for (int x = 0; x < N; ++x) {
        double S[3];
        orc_local_field(L, J, s, x, S);
        orc_or_update(S, &s[3 * x]);
    }
}

/* Initial configuration: mode 0 uniform on the sphere (purpose 4), mode 1
 * all spins (1,0,0) as in the equilibration study of section IV.C. */
void orc_init_spins(int L, double *s, int mode, uint64_t seed, uint32_t sample,
                    uint32_t rep_id)
{
    int N = L * L * L;
    for (int x = 0; x < N; ++x) {
        if (mode == 1) {
            s[3 * x] = 1.0; s[3 * x + 1] = 0.0; s[3 * x + 2] = 0.0;
            continue;
        }
        uint32_t w[4];
        orc_rng_words(seed, sample, (uint32_t)x, rep_id, 0, 4u, w);
        double z = (double)(w[0] >> 8) * 0x1p-23 - 1.0;
        double phi = orc_uniform_phi(w[1]);
        double rho = sqrt(1.0 - z * z);
        s[3 * x] = rho * cos(phi);
        s[3 * x + 1] = rho * sin(phi);
        s[3 * x + 2] = z;
    }
}

/* ------------------------------------------------------------------------ */
/* Round trips (section IV.B): a configuration that has visited the highest */
/* temperature (index 0), then the lowest (index NT-1), completes a round   */
/* trip when it is back at index 0.  rt_state per label: 0 = none yet,      */
/* 1 = last extreme was index 0, 2 = reached index NT-1 after index 0.      */
/* ------------------------------------------------------------------------ */
void orc_roundtrip_update(int NT, const int32_t *label, int32_t *rt_state,
                          int64_t *rt_count)
{
    int top = label[0];
    int bot = label[NT - 1];
    if (rt_state[bot] == 1) rt_state[bot] = 2;
    if (rt_state[top] == 2) { (*rt_count)++; rt_state[top] = 1; }
    else if (rt_state[top] == 0) rt_state[top] = 1;
}

static void swap_configs(int N, double *spins, double *H, int32_t *label, int b)
{
    double *a = spins + (size_t)b * 3 * N, *c = spins + (size_t)(b + 1) * 3 * N;
    for (int n = 0; n < 3 * N; ++n) { double t = a[n]; a[n] = c[n]; c[n] = t; }
    double th = H[b]; H[b] = H[b + 1]; H[b + 1] = th;
    int32_t tl = label[b]; label[b] = label[b + 1]; label[b + 1] = tl;
}

static int accept_metropolis(double lnA, double u) { return lnA >= 0.0 || u < exp(lnA); }

/* ------------------------------------------------------------------------ */
/* Standard exchange (section I, Eq. 1): for the pairs i = 0 .. NT-2 in      */
/* increasing beta, one after the other, accept the swap of the             */
/* configurations at beta_i and beta_{i+1} with probability                  */
/* min[1, exp((beta_{i+1} - beta_i)(H_{i+1} - H_i))].                       */
/* ------------------------------------------------------------------------ */
void orc_exchange_plain(int L, int NT, const double *betas, double *spins,
                        double *H, int32_t *label, int32_t *rt_state,
                        int64_t *rt_count, int64_t *prop, int64_t *acc,
                        uint64_t seed, uint32_t sample, uint32_t copy,
                        uint64_t step)
{
    int N = L * L * L;
    for (int i = 0; i + 1 < NT; ++i) {
        double lnA = (betas[i + 1] - betas[i]) * (H[i + 1] - H[i]);
        uint32_t w[4];
        orc_rng_words(seed, sample, (uint32_t)i, copy, step, 1u, w);
        double u = orc_uniform_u53(w[0], w[1]);
        prop[i]++;
        if (accept_metropolis(lnA, u)) {
            acc[i]++;
            swap_configs(N, spins, H, label, i);
        }
    }
    orc_roundtrip_update(NT, label, rt_state, rt_count);
}

/* ------------------------------------------------------------------------ */
/* Decimation (section III.A).  ln I(beta S)/(4 pi) = ln(sinh R / R),        */
/* R = beta |S| (Eq. HI, with 2c = 4 pi).  ln[2 sinh R] = R + ln[1 - e^-2R]  */
/* (appendix A).                                                            */
/* ------------------------------------------------------------------------ */
double orc_ln_sinhc(double R)
{
    if (R == 0.0) return 0.0;
    if (R < 0.5) return log(sinh(R) / R);
    return R + log1p(-exp(-2.0 * R)) - log(2.0 * R);
}

/* ln of the acceptance ratio of Eq. aswap for decimated colour d: product
 * over x of colour d of I(b2 S1) I(b1 S2) / (I(b1 S1) I(b2 S2)). */
double orc_decimation_lnA(int L, const double *J, const double *s1,
                          const double *s2, int d, double b1, double b2)
{
    int N = L * L * L;
    double lnA = 0.0;
    for (int x = 0; x < N; ++x) {
        if (orc_color(L, x) != d) continue;
        double S1[3], S2[3];
        orc_local_field(L, J, s1, x, S1);
        orc_local_field(L, J, s2, x, S2);
        double a = sqrt(S1[0] * S1[0] + S1[1] * S1[1] + S1[2] * S1[2]);
        double b = sqrt(S2[0] * S2[0] + S2[1] * S2[1] + S2[2] * S2[2]);
        lnA += orc_ln_sinhc(b2 * a) - orc_ln_sinhc(b1 * a) +
               orc_ln_sinhc(b1 * b) - orc_ln_sinhc(b2 * b);
    }
    return lnA;
}

/* Decimation exchange: decimated colour alternates from pair to pair, the
 * first pair's colour is random; on acceptance the decimated sites of both
 * configurations are re-inserted by a heat bath at their new beta, otherwise
 * nothing changes (section III.A, last paragraphs). */
void orc_exchange_decimation(int L, const double *J, int NT, const double *betas,
                             double *spins, double *H, int32_t *label,
                             int32_t *rt_state, int64_t *rt_count, int64_t *prop,
                             int64_t *acc, uint64_t seed, uint32_t sample,
                             uint32_t copy, uint64_t step)
{
    int N = L * L * L;
    uint32_t w[4];
    orc_rng_words(seed, sample, 0u, copy, step, 3u, w);
    int d0 = (int)(w[0] & 1u);
    for (int i = 0; i + 1 < NT; ++i) {
        int d = (d0 + i) & 1;
        double *s1 = spins + (size_t)i * 3 * N;
        double *s2 = spins + (size_t)(i + 1) * 3 * N;
        double lnA = orc_decimation_lnA(L, J, s1, s2, d, betas[i], betas[i + 1]);
        orc_rng_words(seed, sample, (uint32_t)i, copy, step, 1u, w);
        double u = orc_uniform_u53(w[0], w[1]);
        prop[i]++;
        if (accept_metropolis(lnA, u)) {
            acc[i]++;
            swap_configs(N, spins, H, label, i);
            orc_hb_halfsweep(L, J, s1, d, betas[i], seed, sample,
                             copy * (uint32_t)NT + (uint32_t)i, step, 2u);
            orc_hb_halfsweep(L, J, s2, d, betas[i + 1], seed, sample,
                             copy * (uint32_t)NT + (uint32_t)(i + 1), step, 2u);
            H[i] = orc_energy(L, J, s1);
            H[i + 1] = orc_energy(L, J, s2);
        }
    }
    orc_roundtrip_update(NT, label, rt_state, rt_count);
}

/* ------------------------------------------------------------------------ */
/* Cooling and heating (section III.B).                                     */
/* Elementary cooling step at one site: p = S - (S.s) s, alpha = eps |p|,   */
/* s' = s cos(alpha) + p/|p| sin(alpha); it lowers the angle theta between  */
/* s and S by alpha.  Jacobian (measure d cos theta):                       */
/* det J_f = |1 - eps S.s| (cos alpha - cot(theta) sin(alpha)).             */
/* With alpha = eps |S| sin(theta), cot(theta) sin(alpha) =                 */
/* eps (S.s) sin(alpha)/alpha, which is how it is evaluated here.           */
/* ------------------------------------------------------------------------ */
static double sinc(double a) { return (a == 0.0) ? 1.0 : sin(a) / a; }

double orc_cool_site(double eps, const double S[3], double s[3])
{
    double sS = s[0] * S[0] + s[1] * S[1] + s[2] * S[2];
    double p[3] = {S[0] - sS * s[0], S[1] - sS * s[1], S[2] - sS * s[2]};
    double pn = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    double alpha = eps * pn;
    double ca = cos(alpha), sa_over = eps * sinc(alpha); /* sin(alpha)/|p| */
    double j = (1.0 - eps * sS) * (ca - eps * sS * sinc(alpha));
    for (int a = 0; a < 3; ++a) s[a] = s[a] * ca + p[a] * sa_over;
    renormalise(s);
    return log(fabs(j));
}

/* Inverse of the cooling step: theta' given, solve
 * theta - e sin(theta) = theta', e = eps |S| < 1, by Newton's method
 * (section III.B) from theta' + e sin(theta') until the step is below
 * 1e-15 (at most 50 steps), then rotate s' away from S by
 * alpha = theta - theta'.  Returns ln det J_f evaluated at the pre-image. */
double orc_kepler_solve(double e, double thp)
{
    double th = thp + e * sin(thp);
    for (int it = 0; it < 50; ++it) {
        double f = th - e * sin(th) - thp;
        double fp = 1.0 - e * cos(th);
        double d = f / fp;
        th -= d;
        if (th < 0.0) th = 0.0;
        if (th > ORC_PI) th = ORC_PI;
        if (fabs(d) < 1e-15) break;
    }
    return th;
}

double orc_heat_site(double eps, const double S[3], double s[3])
{
    double nS = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
    double sS = s[0] * S[0] + s[1] * S[1] + s[2] * S[2];
    double p[3] = {S[0] - sS * s[0], S[1] - sS * s[1], S[2] - sS * s[2]};
    double pn = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    double e = eps * nS;
    double thp = atan2(pn, sS);
    double th = orc_kepler_solve(e, thp);
    double alpha = th - thp;
    if (pn > 0.0) {
        double f = sin(alpha) / pn;
        for (int a = 0; a < 3; ++a) s[a] = s[a] * cos(alpha) - p[a] * f;
        renormalise(s);
    }
    double c = cos(th);
    double al = e * sin(th);
    double j = (1.0 - e * c) * (cos(al) - e * c * sinc(al));
    return log(fabs(j));
}

/* Cooling sweep C: colour 0 then colour 1.  Returns ln det of its Jacobian. */
double orc_cool_sweep(int L, const double *J, double *s, double eps)
{
    int N = L * L * L;
    double lnJ = 0.0;
    for (int color = 0; color < 2; ++color)
        for (int x = 0; x < N; ++x) {
            if (orc_color(L, x) != color) continue;
            double S[3];
            orc_local_field(L, J, s, x, S);
            lnJ += orc_cool_site(eps, S, &s[3 * x]);
        }
    return lnJ;
}

/* Heating sweep C^-1: colour 1 then colour 0, each the inverse step.
 * Returns ln det J_C evaluated at the result C^-1(s). */
double orc_heat_sweep(int L, const double *J, double *s, double eps)
{
    int N = L * L * L;
    double lnJ = 0.0;
    for (int color = 1; color >= 0; --color)
        for (int x = 0; x < N; ++x) {
            if (orc_color(L, x) != color) continue;
            double S[3];
            orc_local_field(L, J, s, x, S);
            lnJ += orc_heat_site(eps, S, &s[3 * x]);
        }
    return lnJ;
}

/* Test hook, not a reading of the paper: where the acceptance ratio takes
 * the Jacobian of the heated configuration.  0 (the default, used by
 * everything but the power test of the exactness check): ln det J_C at the
 * pre-image C^-1(s2), as the involution requires.  1: at s2 itself, the
 * paper's printed formula read literally.  2: no Jacobian terms at all.
 * Variants 1 and 2 break detailed balance; the test suite shows that its
 * exactness check detects them. */
static int orc_jacobian_variant = 0;

void orc_test_set_jacobian_variant(int v) { orc_jacobian_variant = v; }

/* Cooling/heating exchange of the pair (beta_1 < beta_2): the configuration
 * at beta_1 is cooled and proposed at beta_2, the one at beta_2 is heated
 * and proposed at beta_1.  The map is an involution, so
 * ln A = -b2 H[C s1] - b1 H[C^-1 s2] + b1 H[s1] + b2 H[s2]
 *        + ln det J_C(s1) - ln det J_C(C^-1 s2). */
double orc_coolheat_lnA(int L, const double *J, const double *s1,
                        const double *s2, double H1, double H2, double b1,
                        double b2, double eps, double *t1, double *t2,
                        double *Hc, double *Hh)
{
    int N = L * L * L;
    memcpy(t1, s1, sizeof(double) * 3 * N);
    memcpy(t2, s2, sizeof(double) * 3 * N);
    double lnJ1 = orc_cool_sweep(L, J, t1, eps);
    double lnJ2 = orc_heat_sweep(L, J, t2, eps);
    if (orc_jacobian_variant == 1) {
        /* ln det J_C at s2: cool a copy of s2 and keep only its Jacobian */
        double *tmp = (double *)malloc(sizeof(double) * 3 * N);
        memcpy(tmp, s2, sizeof(double) * 3 * N);
        lnJ2 = orc_cool_sweep(L, J, tmp, eps);
        free(tmp);
    } else if (orc_jacobian_variant == 2) {
        lnJ1 = 0.0;
        lnJ2 = 0.0;
    }
    *Hc = orc_energy(L, J, t1);
    *Hh = orc_energy(L, J, t2);
    return -b2 * (*Hc) - b1 * (*Hh) + b1 * H1 + b2 * H2 + lnJ1 - lnJ2;
}

void orc_exchange_coolheat(int L, const double *J, int NT, const double *betas,
                           const double *eps, double *spins, double *H,
                           int32_t *label, int32_t *rt_state, int64_t *rt_count,
                           int64_t *prop, int64_t *acc, uint64_t seed,
                           uint32_t sample, uint32_t copy, uint64_t step)
{
    int N = L * L * L;
    double *t1 = (double *)malloc(sizeof(double) * 3 * N);
    double *t2 = (double *)malloc(sizeof(double) * 3 * N);
    for (int i = 0; i + 1 < NT; ++i) {
        double *s1 = spins + (size_t)i * 3 * N;
        double *s2 = spins + (size_t)(i + 1) * 3 * N;
        double Hc, Hh;
        double lnA = orc_coolheat_lnA(L, J, s1, s2, H[i], H[i + 1], betas[i],
                                      betas[i + 1], eps[i], t1, t2, &Hc, &Hh);
        uint32_t w[4];
        orc_rng_words(seed, sample, (uint32_t)i, copy, step, 1u, w);
        double u = orc_uniform_u53(w[0], w[1]);
        prop[i]++;
        if (accept_metropolis(lnA, u)) {
            acc[i]++;
            /* C(s1) goes to beta_{i+1}, C^-1(s2) to beta_i; labels follow. */
            memcpy(s1, t2, sizeof(double) * 3 * N);
            memcpy(s2, t1, sizeof(double) * 3 * N);
            H[i] = Hh;
            H[i + 1] = Hc;
            int32_t tl = label[i]; label[i] = label[i + 1]; label[i + 1] = tl;
        }
    }
    free(t1);
    free(t2);
    orc_roundtrip_update(NT, label, rt_state, rt_count);
}

/* ------------------------------------------------------------------------ */
/* Cycles of one sample (section IV): per cycle n_hb heat-                 */
/* bath sweeps and n_or overrelaxation sweeps (each a colour-0 then colour-1 */
/* half sweep) of every replica, then one exchange per chain.  The counter   */
/* `step` advances once per half sweep and once per exchange, shared by all  */
/* chains.  order 0 = checkerboard, 1 = typewriter (statistical only).       */
/* Records H[cycle][copy][b], chi[cycle][b] (if two copies) after the        */
/* exchange.                                                                 */
/* ------------------------------------------------------------------------ */
void orc_pt_run(int L, const double *J, int NT, const double *betas,
                const double *eps, int n_copies, double *spins /* [C][NT][3N] */,
                double *H /* [C][NT] */, int32_t *label /* [C][NT] */,
                int32_t *rt_state /* [C][NT] */, int64_t *rt_count /* [C] */,
                int64_t *prop /* [C][NT-1] */, int64_t *acc /* [C][NT-1] */,
                int n_cycles, int n_hb, int n_or, int mode, int order,
                uint64_t seed, uint32_t sample, uint64_t *step,
                double *H_series, double *chi_series, double *Q_series)
{
    int N = L * L * L;
    size_t rep = (size_t)3 * N;
    for (int cyc = 0; cyc < n_cycles; ++cyc) {
        for (int h = 0; h < n_hb; ++h) {
            if (order == 0) {
                for (int color = 0; color < 2; ++color) {
                    for (int c = 0; c < n_copies; ++c)
                        for (int b = 0; b < NT; ++b)
                            orc_hb_halfsweep(L, J, spins + ((size_t)c * NT + b) * rep,
                                             color, betas[b], seed, sample,
                                             (uint32_t)(c * NT + b), *step, 0u);
                    (*step)++;
                }
            } else {
                for (int c = 0; c < n_copies; ++c)
                    for (int b = 0; b < NT; ++b)
                        orc_hb_sweep_typewriter(L, J, spins + ((size_t)c * NT + b) * rep,
                                                betas[b], seed, sample,
                                                (uint32_t)(c * NT + b), *step);
                (*step) += 2;
            }
        }
        for (int o = 0; o < n_or; ++o) {
            if (order == 0) {
                for (int color = 0; color < 2; ++color) {
                    for (int c = 0; c < n_copies; ++c)
                        for (int b = 0; b < NT; ++b)
                            orc_or_halfsweep(L, J, spins + ((size_t)c * NT + b) * rep,
                                             color);
                    (*step)++;
                }
            } else {
                for (int c = 0; c < n_copies; ++c)
                    for (int b = 0; b < NT; ++b)
                        orc_or_sweep_typewriter(L, J, spins + ((size_t)c * NT + b) * rep);
                (*step) += 2;
            }
        }
        for (int c = 0; c < n_copies; ++c)
            for (int b = 0; b < NT; ++b)
                H[c * NT + b] = orc_energy(L, J, spins + ((size_t)c * NT + b) * rep);
        for (int c = 0; c < n_copies; ++c) {
            double *sp = spins + (size_t)c * NT * rep;
            double *Hc = H + c * NT;
            int32_t *lb = label + c * NT, *rs = rt_state + c * NT;
            int64_t *pr = prop + c * (NT - 1), *ac = acc + c * (NT - 1);
            if (mode == 0)
                orc_exchange_plain(L, NT, betas, sp, Hc, lb, rs, rt_count + c, pr,
                                   ac, seed, sample, (uint32_t)c, *step);
            else if (mode == 1)
                orc_exchange_decimation(L, J, NT, betas, sp, Hc, lb, rs,
                                        rt_count + c, pr, ac, seed, sample,
                                        (uint32_t)c, *step);
            else
                orc_exchange_coolheat(L, J, NT, betas, eps, sp, Hc, lb, rs,
                                      rt_count + c, pr, ac, seed, sample,
                                      (uint32_t)c, *step);
        }
        (*step)++;
        if (H_series)
            for (int n = 0; n < n_copies * NT; ++n)
                H_series[(size_t)cyc * n_copies * NT + n] = H[n];
        if (n_copies == 2 && (chi_series || Q_series)) {
            for (int b = 0; b < NT; ++b) {
                double Q[9];
                double chi = orc_overlap(L, spins + (size_t)b * rep,
                                         spins + ((size_t)NT + b) * rep, Q);
                if (chi_series) chi_series[(size_t)cyc * NT + b] = chi;
                if (Q_series)
                    for (int n = 0; n < 9; ++n)
                        Q_series[((size_t)cyc * NT + b) * 9 + n] = Q[n];
            }
        }
    }
}
