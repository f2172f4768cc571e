// mlp.cu -- the learned ladder: a 4 -> 64 -> 64 -> 2P+1 perceptron that maps a
// sample's description (ln L, beta_min, beta_max, coupling statistic) to the
// shape of its inverse-temperature ladder, the cooling/heating parameter
// along it (section III.B: the optimal epsilon depends on the pair of
// temperatures and falls with beta_{i+1}/beta_i) and the total rejection
// length of the range, which fixes the number of replicas.  It only chooses
// parameters of the tempering; the Markov chain is exact for any ladder.
//
// Weights live in bfloat16 for the forward and backward products (float
// accumulation); an FP32 master copy, the Adam moments and the biases are
// float.  Parameter vector (float): [W1 (64 x 4) | b1 (64) | W2 (64 x 64) |
// b2 (64) | W3 (2P+1 x 64) | b3 (2P+1)], row-major W[out][in].
//
// Outputs z of a row, P knots u_k = k / P:
//   d_k = softplus(z_k) + PT_MLP_SHAPE_FLOOR, f_k = d_k / sum_j d_j, k < P
//   (shape increments; the floor keeps every f_k > 0, so ladders ascend)
//   F(u_k) = sum_{j<k} f_j, F linear between knots; F(u) = u is geometric
//   ln beta(u) = ln beta_min + F(u) ln(beta_max / beta_min)
//   e_k = sigmoid(z_{P+k}),  kappa(u) = kappa_max e(u), e linear between the
//   knot midpoints (k + 1/2) / P and constant beyond the outer ones
//   eps_i = kappa(u at the pair's midpoint) (ln beta_{i+1} - ln beta_i)
//   Lambda = exp(z_{2P}): the sum over pairs of the width sigma of the
//   Gaussian log acceptance ratio; NT = 1 + ceil(Lambda / sigma_target)
//   replicas give every pair the acceptance erfc(sigma_target / 2^{3/2})
// Training loss of a row (targets tf, te, tl):
//   (1/P) sum_k [ (P (f_k - tf_k))^2 + w_kappa (e_k - te_k)^2 ]
//   + (z_{2P} - tl)^2, averaged over the rows.
//
// All kernels are deterministic: gradients are summed per chunk of rows in
// shared memory, then over chunks in a fixed order.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/pt.h"
#include "kernels.h"

namespace {

constexpr int IN = PT_MLP_IN, HID = PT_MLP_HIDDEN;
constexpr int ROWS_PER_CHUNK = 32;
constexpr int MT = 256;  // threads of the backward kernel
constexpr int MAX_KNOTS = PT_MLP_MAX_KNOTS;
constexpr float FLOOR = PT_MLP_SHAPE_FLOOR;

struct Layout {
    int P = 1, N = 2;
    int oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0, total = 0;
    Layout() = default;
    explicit Layout(int knots) {
        P = knots;
        N = 2 * knots + 1;
        oW1 = 0;
        ob1 = oW1 + HID * IN;
        oW2 = ob1 + HID;
        ob2 = oW2 + HID * HID;
        oW3 = ob2 + HID;
        ob3 = oW3 + N * HID;
        total = ob3 + N;
    }
};

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float softplus(float z) { return z > 20.f ? z : log1pf(expf(z)); }
__device__ __forceinline__ float sigm(float z) { return 1.f / (1.f + expf(-z)); }

// Forward pass, one block of 64 threads per row; the post-ReLU activations
// are kept for the backward pass.
__global__ void __launch_bounds__(HID) k_mlp_forward(const float* __restrict__ X, const __nv_bfloat16* __restrict__ Wb,
                                                     const float* __restrict__ prm, Layout ly, int B,
                                                     float* __restrict__ H1, float* __restrict__ H2,
                                                     float* __restrict__ Z) {
    __shared__ float x[IN], h1[HID], h2[HID];
    const int r = blockIdx.x, j = threadIdx.x;
    if (r >= B) return;
    if (j < IN) x[j] = X[(size_t)r * IN + j];
    __syncthreads();
    float a = prm[ly.ob1 + j];
#pragma unroll
    for (int k = 0; k < IN; ++k) a = fmaf(bf(Wb[ly.oW1 + j * IN + k]), x[k], a);
    h1[j] = fmaxf(a, 0.f);
    H1[(size_t)r * HID + j] = h1[j];
    __syncthreads();
    float c = prm[ly.ob2 + j];
#pragma unroll 8
    for (int k = 0; k < HID; ++k) c = fmaf(bf(Wb[ly.oW2 + j * HID + k]), h1[k], c);
    h2[j] = fmaxf(c, 0.f);
    H2[(size_t)r * HID + j] = h2[j];
    __syncthreads();
    for (int n = j; n < ly.N; n += HID) {
        float z = prm[ly.ob3 + n];
#pragma unroll 8
        for (int k = 0; k < HID; ++k) z = fmaf(bf(Wb[ly.oW3 + n * HID + k]), h2[k], z);
        Z[(size_t)r * ly.N + n] = z;
    }
}

// Loss of every row and dL/dz (the 1/B of the batch mean included).
__global__ void k_mlp_loss(const float* __restrict__ Z, const float* __restrict__ T, int B, int P, float w_kappa,
                           float* __restrict__ GZ, float* __restrict__ row_loss) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= B) return;
    const int N = 2 * P + 1;
    const float* z = Z + (size_t)r * N;
    const float* t = T + (size_t)r * N;
    float* g = GZ + (size_t)r * N;
    float S = 0.f;
    for (int i = 0; i < P; ++i) S += softplus(z[i]) + FLOOR;
    const float Pf = (float)P, scale = 1.f / (Pf * (float)B);
    float loss = 0.f, dot = 0.f;
    for (int i = 0; i < P; ++i) {
        const float f = (softplus(z[i]) + FLOOR) / S;
        const float d = Pf * (f - t[i]);
        loss += d * d;
        const float df = 2.f * Pf * d * scale;  // dL/df_i
        dot += df * f;
        g[i] = df;
    }
    // f_i = d_i / S, d_i = softplus(z_i) + floor  =>  dL/dd_i = (dL/df_i - sum_k dL/df_k f_k) / S, and
    // d softplus(z) / dz = sigmoid(z)
    for (int i = 0; i < P; ++i) g[i] = (g[i] - dot) / S * sigm(z[i]);
    for (int i = 0; i < P; ++i) {
        const float e = sigm(z[P + i]);
        const float d = e - t[P + i];
        loss += w_kappa * d * d;
        g[P + i] = 2.f * w_kappa * d * scale * e * (1.f - e);
    }
    const float dl = z[2 * P] - t[2 * P];
    g[2 * P] = 2.f * dl / (float)B;
    row_loss[r] = loss / Pf + dl * dl;
}

// Backward pass over a chunk of rows; the chunk's parameter gradient is
// accumulated in shared memory, every entry owned by one thread.
__global__ void __launch_bounds__(MT) k_mlp_backward(const float* __restrict__ X, const __nv_bfloat16* __restrict__ Wb,
                                                     Layout ly, int B, const float* __restrict__ H1,
                                                     const float* __restrict__ H2, const float* __restrict__ GZ,
                                                     float* __restrict__ Gpart) {
    extern __shared__ float sg[];  // ly.total floats
    __shared__ float gz[2 * MAX_KNOTS + 1], gz2[HID], gz1[HID], h1[HID], h2[HID], x[IN];
    const int tid = threadIdx.x, N = ly.N;
    for (int p = tid; p < ly.total; p += MT) sg[p] = 0.f;
    const int r0 = blockIdx.x * ROWS_PER_CHUNK;
    const int r1 = min(B, r0 + ROWS_PER_CHUNK);
    for (int r = r0; r < r1; ++r) {
        __syncthreads();
        for (int n = tid; n < N; n += MT) gz[n] = GZ[(size_t)r * N + n];
        if (tid < HID) {
            h1[tid] = H1[(size_t)r * HID + tid];
            h2[tid] = H2[(size_t)r * HID + tid];
        }
        if (tid < IN) x[tid] = X[(size_t)r * IN + tid];
        __syncthreads();
        if (tid < HID) {
            float a = 0.f;
            for (int n = 0; n < N; ++n) a = fmaf(bf(Wb[ly.oW3 + n * HID + tid]), gz[n], a);
            gz2[tid] = h2[tid] > 0.f ? a : 0.f;
        }
        __syncthreads();
        if (tid < HID) {
            float a = 0.f;
#pragma unroll 8
            for (int j = 0; j < HID; ++j) a = fmaf(bf(Wb[ly.oW2 + j * HID + tid]), gz2[j], a);
            gz1[tid] = h1[tid] > 0.f ? a : 0.f;
        }
        __syncthreads();
        for (int q = tid; q < N * HID; q += MT) sg[ly.oW3 + q] += gz[q / HID] * h2[q % HID];
        for (int n = tid; n < N; n += MT) sg[ly.ob3 + n] += gz[n];
        for (int q = tid; q < HID * HID; q += MT) sg[ly.oW2 + q] += gz2[q / HID] * h1[q % HID];
        for (int q = tid; q < HID; q += MT) sg[ly.ob2 + q] += gz2[q];
        for (int q = tid; q < HID * IN; q += MT) sg[ly.oW1 + q] += gz1[q / IN] * x[q % IN];
        for (int q = tid; q < HID; q += MT) sg[ly.ob1 + q] += gz1[q];
    }
    __syncthreads();
    for (int p = tid; p < ly.total; p += MT) Gpart[(size_t)blockIdx.x * ly.total + p] = sg[p];
}

__global__ void k_mlp_reduce(const float* __restrict__ Gpart, int chunks, int total, float* __restrict__ G) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= total) return;
    float s = 0.f;
    for (int c = 0; c < chunks; ++c) s += Gpart[(size_t)c * total + p];
    G[p] = s;
}

// One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on the
// master weights, then the bfloat16 copy.
__global__ void k_mlp_adam(float* __restrict__ prm, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ G, int total, float lr, float b1c, float b2c,
                           __nv_bfloat16* __restrict__ Wb) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= total) return;
    const float g = G[p];
    const float mm = 0.9f * m[p] + 0.1f * g;
    const float vv = 0.999f * v[p] + 0.001f * g * g;
    m[p] = mm;
    v[p] = vv;
    const float w = prm[p] - lr * (mm / b1c) / (sqrtf(vv / b2c) + 1e-8f);
    prm[p] = w;
    Wb[p] = __float2bfloat16_rn(w);
}

__global__ void k_mlp_cast(const float* __restrict__ prm, int total, __nv_bfloat16* __restrict__ Wb) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < total) Wb[p] = __float2bfloat16_rn(prm[p]);
}

// Ladder and per-pair epsilon of every row from its outputs z; rows with
// n_temps <= 0 take the replica count from the predicted rejection length.
__global__ void k_mlp_decode(const float* __restrict__ Z, int B, int P, const double* __restrict__ bmin,
                             const double* __restrict__ bmax, int* __restrict__ n_temps, int stride,
                             float kappa_max, double sigma_target, double* __restrict__ betas,
                             float* __restrict__ eps) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= B) return;
    const float* z = Z + (size_t)r * (2 * P + 1);
    double F[MAX_KNOTS + 1], e[MAX_KNOTS];
    double S = 0.0;
    for (int k = 0; k < P; ++k) S += (double)(softplus(z[k]) + FLOOR);
    F[0] = 0.0;
    for (int k = 0; k < P; ++k) {
        F[k + 1] = F[k] + (double)(softplus(z[k]) + FLOOR) / S;
        e[k] = (double)sigm(z[P + k]);
    }
    F[P] = 1.0;
    int NT = n_temps[r];
    if (NT <= 0) {
        const double want = 1.0 + ceil(exp((double)z[2 * P]) / sigma_target);
        NT = (int)fmin(fmax(want, 2.0), (double)stride);
        n_temps[r] = NT;
    }
    const double lb0 = log(bmin[r]), lb1 = log(bmax[r]), span = lb1 - lb0;
    double* out = betas + (size_t)r * stride;
    float* ep = eps + (size_t)r * (stride - 1);
    double prev = lb0;
    out[0] = bmin[r];
    for (int i = 1; i < NT; ++i) {
        double lb;
        if (i == NT - 1) {
            lb = lb1;
            out[i] = bmax[r];
        } else {
            const double uP = (double)i / (double)(NT - 1) * (double)P;
            const int k = min((int)uP, P - 1);
            lb = lb0 + span * (F[k] + (uP - (double)k) * (F[k + 1] - F[k]));
            out[i] = exp(lb);
        }
        // kappa at the pair's midpoint, linear between knot midpoints
        const double mP = ((double)i - 0.5) / (double)(NT - 1) * (double)P - 0.5;
        double ev;
        if (mP <= 0.0) ev = e[0];
        else if (mP >= (double)(P - 1)) ev = e[P - 1];
        else {
            const int k = (int)mP;
            ev = e[k] + (mP - (double)k) * (e[k + 1] - e[k]);
        }
        ep[i - 1] = (float)((double)kappa_max * ev * (lb - prev));
        prev = lb;
    }
}

// splitmix64 (Steele, Lea and Flood 2014) for the deterministic initialisation.
uint64_t splitmix(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

struct pt_mlp {
    Layout ly;
    cudaStream_t stream = nullptr;
    float *prm = nullptr, *m = nullptr, *v = nullptr, *G = nullptr;
    __nv_bfloat16* Wb = nullptr;
    int t = 0;  // Adam steps taken
    int cap = 0, cap_nt = 0;
    float *X = nullptr, *T = nullptr, *H1 = nullptr, *H2 = nullptr, *Z = nullptr, *GZ = nullptr, *RL = nullptr,
          *Gpart = nullptr, *eps = nullptr;
    double *bmin = nullptr, *bmax = nullptr, *betas = nullptr;
    int* nt = nullptr;
    std::vector<void*> owned;
};

namespace {

#define MK(call)                                                              \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) {                                              \
            char b_[256];                                                     \
            snprintf(b_, sizeof b_, "%s: %s", #call, cudaGetErrorString(e_)); \
            ptk::set_last_error(b_);                                          \
            return PT_ERR_CUDA;                                               \
        }                                                                     \
    } while (0)

pt_status merr(pt_status st, const char* msg) {
    ptk::set_last_error(msg);
    return st;
}

template <typename X>
pt_status dev_alloc(pt_mlp* h, X** p, size_t n) {
    MK(cudaMalloc((void**)p, sizeof(X) * (n ? n : 1)));
    h->owned.push_back(*p);
    return PT_OK;
}

template <typename X>
pt_status dev_realloc(pt_mlp* h, X** p, size_t n) {
    if (*p) {
        for (auto& q : h->owned)
            if (q == *p) q = nullptr;
        MK(cudaFree(*p));
        *p = nullptr;
    }
    return dev_alloc(h, p, n);
}

pt_status ensure_batch(pt_mlp* h, int B) {
    if (B <= h->cap) return PT_OK;
    MK(cudaStreamSynchronize(h->stream));
    const size_t N = h->ly.N, chunks = (B + ROWS_PER_CHUNK - 1) / ROWS_PER_CHUNK;
    pt_status st = PT_OK;
    if (st == PT_OK) st = dev_realloc(h, &h->X, (size_t)B * IN);
    if (st == PT_OK) st = dev_realloc(h, &h->T, (size_t)B * N);
    if (st == PT_OK) st = dev_realloc(h, &h->H1, (size_t)B * HID);
    if (st == PT_OK) st = dev_realloc(h, &h->H2, (size_t)B * HID);
    if (st == PT_OK) st = dev_realloc(h, &h->Z, (size_t)B * N);
    if (st == PT_OK) st = dev_realloc(h, &h->GZ, (size_t)B * N);
    if (st == PT_OK) st = dev_realloc(h, &h->RL, (size_t)B);
    if (st == PT_OK) st = dev_realloc(h, &h->Gpart, chunks * h->ly.total);
    if (st == PT_OK) st = dev_realloc(h, &h->bmin, (size_t)B);
    if (st == PT_OK) st = dev_realloc(h, &h->bmax, (size_t)B);
    if (st == PT_OK) st = dev_realloc(h, &h->nt, (size_t)B);
    if (st != PT_OK) return st;
    h->cap = B;
    h->cap_nt = 0;  // ladder outputs are sized on demand
    return PT_OK;
}

pt_status forward(pt_mlp* h, int B, const float* x) {
    MK(cudaMemcpyAsync(h->X, x, sizeof(float) * B * IN, cudaMemcpyHostToDevice, h->stream));
    k_mlp_forward<<<B, HID, 0, h->stream>>>(h->X, h->Wb, h->prm, h->ly, B, h->H1, h->H2, h->Z);
    MK(cudaGetLastError());
    return PT_OK;
}

pt_status loss_grad(pt_mlp* h, int B, const float* x, const float* target, float w_kappa) {
    const Layout& L = h->ly;
    pt_status st = forward(h, B, x);
    if (st != PT_OK) return st;
    MK(cudaMemcpyAsync(h->T, target, sizeof(float) * B * L.N, cudaMemcpyHostToDevice, h->stream));
    k_mlp_loss<<<(B + 127) / 128, 128, 0, h->stream>>>(h->Z, h->T, B, L.P, w_kappa, h->GZ, h->RL);
    MK(cudaGetLastError());
    const int chunks = (B + ROWS_PER_CHUNK - 1) / ROWS_PER_CHUNK;
    const size_t smem = sizeof(float) * L.total;
    MK(ptk::ensure_smem((const void*)k_mlp_backward, smem));
    k_mlp_backward<<<chunks, MT, smem, h->stream>>>(h->X, h->Wb, L, B, h->H1, h->H2, h->GZ, h->Gpart);
    MK(cudaGetLastError());
    k_mlp_reduce<<<(L.total + 255) / 256, 256, 0, h->stream>>>(h->Gpart, chunks, L.total, h->G);
    MK(cudaGetLastError());
    return PT_OK;
}

pt_status read_loss(pt_mlp* h, int B, float* loss) {
    std::vector<float> rl(B);
    MK(cudaMemcpyAsync(rl.data(), h->RL, sizeof(float) * B, cudaMemcpyDeviceToHost, h->stream));
    MK(cudaStreamSynchronize(h->stream));
    double s = 0.0;
    for (float v : rl) s += v;
    *loss = (float)(s / B);
    return PT_OK;
}

bool all_finite(const float* p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

pt_status check_targets(pt_mlp* h, int batch, const float* x, const float* target, float w_kappa) {
    if (!all_finite(x, (size_t)batch * IN)) return merr(PT_ERR_ARG, "non-finite feature");
    if (!all_finite(target, (size_t)batch * h->ly.N)) return merr(PT_ERR_ARG, "non-finite target");
    if (!(w_kappa >= 0.f) || !std::isfinite(w_kappa)) return merr(PT_ERR_ARG, "w_kappa must be finite and >= 0");
    return PT_OK;
}

}  // namespace

extern "C" {

pt_status pt_mlp_create(pt_mlp_handle* out, int n_knots, uint64_t seed, void* stream) {
    if (!out) return merr(PT_ERR_ARG, "NULL out");
    *out = nullptr;
    if (n_knots < 1 || n_knots > MAX_KNOTS) return merr(PT_ERR_ARG, "n_knots must be in [1, PT_MLP_MAX_KNOTS]");
    pt_mlp* h = new (std::nothrow) pt_mlp();
    if (!h) return merr(PT_ERR_NOMEM, "host allocation failed");
    h->ly = Layout(n_knots);
    h->stream = (cudaStream_t)stream;
    const int total = h->ly.total;
    pt_status st = dev_alloc(h, &h->prm, total);
    if (st == PT_OK) st = dev_alloc(h, &h->m, total);
    if (st == PT_OK) st = dev_alloc(h, &h->v, total);
    if (st == PT_OK) st = dev_alloc(h, &h->G, total);
    if (st == PT_OK) st = dev_alloc(h, &h->Wb, total);
    if (st != PT_OK) {
        pt_mlp_destroy(h);
        return st;
    }
    // uniform(-1, 1) / sqrt(fan_in) weights, zero biases; the last layer is
    // scaled down so that a fresh net starts near F(u) = u (geometric).
    std::vector<float> init(total, 0.f);
    uint64_t s = seed;
    auto uni = [&]() { return (double)(splitmix(s) >> 11) * 0x1p-53 * 2.0 - 1.0; };
    const Layout& L = h->ly;
    for (int q = 0; q < HID * IN; ++q) init[L.oW1 + q] = (float)(uni() / std::sqrt((double)IN));
    for (int q = 0; q < HID * HID; ++q) init[L.oW2 + q] = (float)(uni() / std::sqrt((double)HID));
    for (int q = 0; q < L.N * HID; ++q) init[L.oW3 + q] = (float)(0.01 * uni() / std::sqrt((double)HID));
    st = pt_mlp_set_params(h, init.data());
    if (st != PT_OK) {
        pt_mlp_destroy(h);
        return st;
    }
    *out = h;
    return PT_OK;
}

int pt_mlp_num_params(pt_mlp_handle h) { return h ? h->ly.total : 0; }

pt_status pt_mlp_set_params(pt_mlp_handle h, const float* params) {
    if (!h || !params) return merr(PT_ERR_ARG, "NULL argument");
    const int total = h->ly.total;
    if (!all_finite(params, total)) return merr(PT_ERR_ARG, "non-finite parameter");
    MK(cudaMemcpyAsync(h->prm, params, sizeof(float) * total, cudaMemcpyHostToDevice, h->stream));
    MK(cudaMemsetAsync(h->m, 0, sizeof(float) * total, h->stream));
    MK(cudaMemsetAsync(h->v, 0, sizeof(float) * total, h->stream));
    k_mlp_cast<<<(total + 255) / 256, 256, 0, h->stream>>>(h->prm, total, h->Wb);
    MK(cudaGetLastError());
    MK(cudaStreamSynchronize(h->stream));
    h->t = 0;
    return PT_OK;
}

pt_status pt_mlp_get_params(pt_mlp_handle h, float* params, uint16_t* bf16) {
    if (!h) return merr(PT_ERR_ARG, "NULL handle");
    const int total = h->ly.total;
    if (params) MK(cudaMemcpyAsync(params, h->prm, sizeof(float) * total, cudaMemcpyDeviceToHost, h->stream));
    if (bf16) MK(cudaMemcpyAsync(bf16, h->Wb, sizeof(uint16_t) * total, cudaMemcpyDeviceToHost, h->stream));
    MK(cudaStreamSynchronize(h->stream));
    return PT_OK;
}

pt_status pt_mlp_forward(pt_mlp_handle h, int batch, const float* x, float* z) {
    if (!h || !x || !z || batch < 1) return merr(PT_ERR_ARG, "bad argument");
    if (!all_finite(x, (size_t)batch * IN)) return merr(PT_ERR_ARG, "non-finite feature");
    pt_status st = ensure_batch(h, batch);
    if (st == PT_OK) st = forward(h, batch, x);
    if (st != PT_OK) return st;
    MK(cudaMemcpyAsync(z, h->Z, sizeof(float) * batch * h->ly.N, cudaMemcpyDeviceToHost, h->stream));
    MK(cudaStreamSynchronize(h->stream));
    return PT_OK;
}

pt_status pt_mlp_loss_grad(pt_mlp_handle h, int batch, const float* x, const float* target, float w_kappa,
                           float* loss, float* grad) {
    if (!h || !x || !target || batch < 1) return merr(PT_ERR_ARG, "bad argument");
    pt_status st = check_targets(h, batch, x, target, w_kappa);
    if (st == PT_OK) st = ensure_batch(h, batch);
    if (st == PT_OK) st = loss_grad(h, batch, x, target, w_kappa);
    if (st != PT_OK) return st;
    if (grad) MK(cudaMemcpyAsync(grad, h->G, sizeof(float) * h->ly.total, cudaMemcpyDeviceToHost, h->stream));
    if (loss) return read_loss(h, batch, loss);
    MK(cudaStreamSynchronize(h->stream));
    return PT_OK;
}

pt_status pt_mlp_train(pt_mlp_handle h, int batch, const float* x, const float* target, float w_kappa, int steps,
                       float lr, float* losses) {
    if (!h || !x || !target || batch < 1 || steps < 0 || !(lr > 0.f) || !std::isfinite(lr))
        return merr(PT_ERR_ARG, "bad argument");
    pt_status st = check_targets(h, batch, x, target, w_kappa);
    if (st == PT_OK) st = ensure_batch(h, batch);
    if (st != PT_OK) return st;
    const int total = h->ly.total;
    for (int k = 0; k < steps; ++k) {
        st = loss_grad(h, batch, x, target, w_kappa);
        if (st != PT_OK) return st;
        h->t += 1;
        const float b1c = 1.f - powf(0.9f, (float)h->t), b2c = 1.f - powf(0.999f, (float)h->t);
        k_mlp_adam<<<(total + 255) / 256, 256, 0, h->stream>>>(h->prm, h->m, h->v, h->G, total, lr, b1c, b2c, h->Wb);
        MK(cudaGetLastError());
        if (losses) {
            st = read_loss(h, batch, &losses[k]);
            if (st != PT_OK) return st;
        }
    }
    MK(cudaStreamSynchronize(h->stream));
    return PT_OK;
}

pt_status pt_mlp_ladder(pt_mlp_handle h, int batch, const float* x, const double* beta_min, const double* beta_max,
                        int* n_temps, int stride, float kappa_max, double sigma_target, double* betas, float* eps) {
    if (!h || !x || !beta_min || !beta_max || !n_temps || !betas || !eps || batch < 1 || stride < 2)
        return merr(PT_ERR_ARG, "bad argument");
    if (!all_finite(x, (size_t)batch * IN)) return merr(PT_ERR_ARG, "non-finite feature");
    if (!(kappa_max >= 0.f) || !std::isfinite(kappa_max)) return merr(PT_ERR_ARG, "kappa_max must be finite and >= 0");
    bool choose = false;
    for (int r = 0; r < batch; ++r) {
        if (!(beta_min[r] > 0.0) || !(beta_max[r] > beta_min[r]) || !std::isfinite(beta_max[r]))
            return merr(PT_ERR_ARG, "need 0 < beta_min < beta_max < inf");
        if (n_temps[r] == 1 || n_temps[r] > stride) return merr(PT_ERR_ARG, "need n_temps <= 0 or 2 <= n_temps <= stride");
        choose |= n_temps[r] <= 0;
    }
    if (choose && !(sigma_target > 0.0 && std::isfinite(sigma_target)))
        return merr(PT_ERR_ARG, "sigma_target must be finite and > 0 when a row chooses its replica count");
    pt_status st = ensure_batch(h, batch);
    if (st != PT_OK) return st;
    if (stride > h->cap_nt) {
        MK(cudaStreamSynchronize(h->stream));
        st = dev_realloc(h, &h->betas, (size_t)h->cap * stride);
        if (st == PT_OK) st = dev_realloc(h, &h->eps, (size_t)h->cap * (stride - 1));
        if (st != PT_OK) return st;
        h->cap_nt = stride;
    }
    st = forward(h, batch, x);
    if (st != PT_OK) return st;
    MK(cudaMemcpyAsync(h->bmin, beta_min, sizeof(double) * batch, cudaMemcpyHostToDevice, h->stream));
    MK(cudaMemcpyAsync(h->bmax, beta_max, sizeof(double) * batch, cudaMemcpyHostToDevice, h->stream));
    MK(cudaMemcpyAsync(h->nt, n_temps, sizeof(int) * batch, cudaMemcpyHostToDevice, h->stream));
    MK(cudaMemsetAsync(h->betas, 0, sizeof(double) * batch * stride, h->stream));
    MK(cudaMemsetAsync(h->eps, 0, sizeof(float) * batch * (stride - 1), h->stream));
    k_mlp_decode<<<(batch + 63) / 64, 64, 0, h->stream>>>(h->Z, batch, h->ly.P, h->bmin, h->bmax, h->nt, stride,
                                                           kappa_max, choose ? sigma_target : 1.0, h->betas, h->eps);
    MK(cudaGetLastError());
    MK(cudaMemcpyAsync(n_temps, h->nt, sizeof(int) * batch, cudaMemcpyDeviceToHost, h->stream));
    MK(cudaMemcpyAsync(betas, h->betas, sizeof(double) * batch * stride, cudaMemcpyDeviceToHost, h->stream));
    MK(cudaMemcpyAsync(eps, h->eps, sizeof(float) * batch * (stride - 1), cudaMemcpyDeviceToHost, h->stream));
    MK(cudaStreamSynchronize(h->stream));
    return PT_OK;
}

pt_status pt_mlp_destroy(pt_mlp_handle h) {
    if (!h) return PT_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    for (void* p : h->owned)
        if (p) cudaFree(p);
    delete h;
    return PT_OK;
}

}  // extern "C"
