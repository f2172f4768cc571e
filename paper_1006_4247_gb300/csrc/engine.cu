// engine.cu -- host side of the C ABI declared in include/pt.h: validation,
// batch descriptors, device memory, launch sequences, observables, checkpoint.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/pt.h"
#include "kernels.h"
#include "pt_types.h"

using namespace ptk;

namespace {

thread_local char g_err[1024] = "";

pt_status fail(pt_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(PT_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                              \
    } while (0)

FastDiv make_fastdiv(uint32_t d) {
    FastDiv f{d, 0u, 0u, 0u};
    if (d <= 1) return f;  // m == 0 flags d == 1
    uint32_t l = 0;
    while ((1ull << l) < d) ++l;
    const unsigned __int128 num = (unsigned __int128)1 << (31 + l);
    f.m = (uint32_t)((num + d - 1) / d);
    f.s = l - 1;
    return f;
}

constexpr int kMaxNT = 512;  // must match the exchange kernels' shared-memory limit

// Sites per thread of the half sweep: 16-byte vectors where the row length
// L/2 allows them (float4 / double2), else 8-byte, else scalar.
int vec_width(int hL, bool fp64) {
    if (!fp64 && hL % 4 == 0) return 4;
    if (hL % 2 == 0) return 2;
    return 1;
}

}  // namespace

void ptk::set_last_error(const char* msg) { snprintf(g_err, sizeof g_err, "%s", msg); }

cudaError_t ptk::ensure_smem(const void* kernel, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    std::lock_guard<std::mutex> lock(mu);
    size_t& have = done[{kernel, dev}];
    if (bytes <= have) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) have = bytes;
    return e;
}

struct pt_engine {
    int S = 0, C = 0;
    bool fp64 = false;
    uint64_t seed = 0;
    int start = 0;
    cudaStream_t stream = nullptr;
    pt_alloc_fn alloc = nullptr;
    pt_free_fn freefn = nullptr;
    void* actx = nullptr;

    std::vector<int> L, NT;
    std::vector<SampleDesc> samples;
    std::vector<ChainDesc> chains;
    std::vector<int4> reps;
    std::vector<int2> tiles;          // half-sweep tiles, grouped by vector class
    std::vector<int> q_sample;
    std::vector<long long> chain_off;
    std::vector<float> maxsumJ;       // per sample: max_x sum of |J| over the 6 bonds
    std::vector<float> eps_host;      // last cooling parameters
    size_t pool_elems = 0, J_elems = 0;
    int R = 0, P = 0, T = 0, sumNT = 0, sumEps = 0;
    bool energy_valid = false;
    int policy = PT_POLICY_AUTO;
    bool all_resident = false;        // every sample fits the resident kernel
    bool any_streaming = true;        // some sample runs streaming half sweeps
    bool all_tma = false;             // every sample fits the bulk-copy half sweep
    std::vector<int4> tma_items;
    std::vector<int> stile_idx;       // streaming subset of `tiles`
    std::vector<int> res_reps;        // replicas of resident samples
    std::vector<int> tuned_vec;       // per sample: vector width chosen by pt_autotune (0: default)
    std::vector<int> tuned_res;       // per sample: -1 default, 0 streaming, 1 resident, 2 narrow clusters (pt_autotune)
    bool narrow_default = false;      // PT_CL_NARROW=1 at creation: narrow clusters unless tuned otherwise
    size_t tile_cap = 0;              // capacity of the tile and partial arrays
    int* d_stiles = nullptr;
    int* d_res_reps = nullptr;
    int* d_nor = nullptr;
    std::vector<int> nor_host;        // per-sample overrelaxation counts last uploaded
    // pinned staging buffers for host parameters (two, used in turn; the
    // event of a buffer marks the end of its last copy)
    struct Staging { void* host = nullptr; size_t bytes = 0; cudaEvent_t ev = nullptr; };
    Staging stage[2];
    int* err_host = nullptr;          // pinned copy of the device error word (read by sync)
    int stage_next = 0;
    // captured update cycle (pt_cycles)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<long long> graph_key;
    long long graph_launches[PT_KERNEL_KINDS] = {0};
    int graph_steps = 0;
    int max_half = 0;
    uint64_t step_host = 0;           // mirror of the device step counter

    std::vector<void*> owned;
    DevBatch d{};

    // per-kernel-class accounting (pt_profile)
    bool profiling = false;
    long long launches[PT_KERNEL_KINDS] = {0};
    struct Rec { int kind; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> ev_pool;
    cudaEvent_t ev_get() {
        if (!ev_pool.empty()) { cudaEvent_t v = ev_pool.back(); ev_pool.pop_back(); return v; }
        cudaEvent_t v = nullptr;
        if (cudaEventCreate(&v) != cudaSuccess) return nullptr;
        return v;
    }

    size_t esz() const { return fp64 ? sizeof(double) : sizeof(float); }

    pt_status dalloc(void** p, size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        if (bytes == 0) bytes = 256;
        if (alloc) {
            *p = alloc(bytes, actx);
            if (!*p) return fail(PT_ERR_NOMEM, "allocator callback returned NULL for %zu bytes", bytes);
        } else {
            cudaError_t e = cudaMalloc(p, bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(e == cudaErrorMemoryAllocation ? PT_ERR_NOMEM : PT_ERR_CUDA,
                            "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
            }
        }
        owned.push_back(*p);
        return PT_OK;
    }

    void release() {
        if (stream) cudaStreamSynchronize(stream); else cudaDeviceSynchronize();
        for (Staging& st : stage) {
            if (st.host) cudaFreeHost(st.host);
            if (st.ev) cudaEventDestroy(st.ev);
            st = Staging();
        }
        if (err_host) cudaFreeHost(err_host);
        err_host = nullptr;
        if (graph_exec) cudaGraphExecDestroy(graph_exec);
        if (graph) cudaGraphDestroy(graph);
        graph_exec = nullptr;
        graph = nullptr;
        for (Rec& r : recs) { ev_pool.push_back(r.a); ev_pool.push_back(r.b); }
        recs.clear();
        for (cudaEvent_t v : ev_pool) if (v) cudaEventDestroy(v);
        ev_pool.clear();
        for (void* p : owned) {
            if (freefn) freefn(p, actx);
            else cudaFree(p);
        }
        owned.clear();
    }
};

namespace {

template <typename X>
pt_status upload(pt_engine* e, X** dst, const std::vector<X>& v) {
    pt_status st = e->dalloc((void**)dst, sizeof(X) * (v.empty() ? 1 : v.size()));
    if (st != PT_OK) return st;
    if (!v.empty())
        CK(cudaMemcpyAsync(*dst, v.data(), sizeof(X) * v.size(), cudaMemcpyHostToDevice, e->stream));
    return PT_OK;
}

// Natural order [N][3] <-> colour-split [c][a][h] of one buffer.
template <typename X>
void natural_to_split(int L, const double* xyz, X* buf) {
    const int N = L * L * L, half = N / 2, hL = L / 2;
    for (int x = 0; x < N; ++x) {
        const int i = x % L, j = (x / L) % L, k = x / (L * L);
        const int c = (i + j + k) & 1;
        const int h = (i >> 1) + hL * (j + L * k);
        for (int a = 0; a < 3; ++a) buf[(size_t)c * 3 * half + (size_t)a * half + h] = (X)xyz[3 * x + a];
    }
}

template <typename X>
void split_to_natural(int L, const X* buf, double* xyz) {
    const int N = L * L * L, half = N / 2, hL = L / 2;
    for (int x = 0; x < N; ++x) {
        const int i = x % L, j = (x / L) % L, k = x / (L * L);
        const int c = (i + j + k) & 1;
        const int h = (i >> 1) + hL * (j + L * k);
        for (int a = 0; a < 3; ++a) xyz[3 * x + a] = (double)buf[(size_t)c * 3 * half + (size_t)a * half + h];
    }
}

// Run a launcher, count its kernels under `kind` and, while profiling,
// bracket it with events on the engine's stream.
template <class F>
pt_status run(pt_engine* e, int kind, int n_kernels, F&& launcher) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (e->profiling) {
        a = e->ev_get();
        b = e->ev_get();
        if (!a || !b) return fail(PT_ERR_CUDA, "cudaEventCreate failed");
        CK(cudaEventRecord(a, e->stream));
    }
    CK(launcher());
    e->launches[kind] += n_kernels;
    if (e->profiling) {
        CK(cudaEventRecord(b, e->stream));
        e->recs.push_back({kind, a, b});
    }
    return PT_OK;
}

#define RUN(kind, n, expr)                                               \
    do {                                                                 \
        pt_status st_ = run(e, kind, n, [&]() { return (expr); });       \
        if (st_ != PT_OK) return st_;                                    \
    } while (0)

// Copy host data to the device on the engine's stream without waiting: the
// bytes go through a pinned staging buffer, so the caller may reuse its array
// as soon as this returns.
pt_status stage_copy(pt_engine* e, void* dst, const void* src, size_t bytes) {
    pt_engine::Staging& st = e->stage[e->stage_next];
    e->stage_next ^= 1;
    if (st.ev) CK(cudaEventSynchronize(st.ev));
    else CK(cudaEventCreateWithFlags(&st.ev, cudaEventDisableTiming));
    if (st.bytes < bytes) {
        if (st.host) cudaFreeHost(st.host);
        st.host = nullptr;
        st.bytes = 0;
        CK(cudaMallocHost(&st.host, bytes));
        st.bytes = bytes;
    }
    std::memcpy(st.host, src, bytes);
    CK(cudaMemcpyAsync(dst, st.host, bytes, cudaMemcpyHostToDevice, e->stream));
    CK(cudaEventRecord(st.ev, e->stream));
    return PT_OK;
}

pt_status compute_energy(pt_engine* e) {
    RUN(PT_KERNEL_ENERGY, energy_launch_count(e->d, true), launch_energy(e->d, e->fp64, true, e->stream));
    RUN(PT_KERNEL_ENERGY, 1, launch_energy_finalize(e->d, true, e->stream));
    e->energy_valid = true;
    return PT_OK;
}

// Which path each sample takes: resident when the policy allows it and the
// replica fits (or pt_autotune chose it), else streaming half sweeps.
void choose_paths(pt_engine* e) {
    e->all_resident = true;
    for (size_t s = 0; s < e->samples.size(); ++s) {
        SampleDesc& sd = e->samples[s];
        const int def_vec = vec_width(sd.hL, e->fp64);
        const int vec = (!e->tuned_vec.empty() && e->tuned_vec[s] > 0) ? e->tuned_vec[s] : def_vec;
        const bool fits = resident_cluster(sd, e->fp64, vec) > 0 || resident_cluster(sd, e->fp64, def_vec) > 0;
        e->all_resident = e->all_resident && fits;
        bool res;
        if (e->policy == PT_POLICY_STREAMING) res = false;
        else if (e->policy == PT_POLICY_RESIDENT) res = fits;
        else res = (!e->tuned_res.empty() && e->tuned_res[s] >= 0) ? (e->tuned_res[s] >= 1 && fits) : fits;
        sd.vec = res ? (resident_cluster(sd, e->fp64, vec) > 0 ? vec : def_vec) : vec;
        sd.resident = res ? resident_cluster(sd, e->fp64, sd.vec) : 0;  // CTAs per replica
        sd.narrow = 0;
        const bool tuned = !e->tuned_res.empty() && e->tuned_res[s] >= 0;
        if (res && (tuned ? e->tuned_res[s] == 2 : e->narrow_default)) {
            const int cn = resident_cluster_narrow(sd, e->fp64, sd.vec);
            if (cn > 0) {
                sd.resident = cn;
                sd.narrow = 1;
            }
        }
        sd.tiles_per_rep = (sd.half + TILE * sd.vec - 1) / (TILE * sd.vec);
    }
}

// (Re)build the tile lists (all samples grouped by vector width, and the
// streaming subset), the resident replica list, and upload them with the
// sample descriptors.
pt_status rebuild_lists(pt_engine* e) {
    const int widths[3] = {4, 2, 1};
    e->tiles.clear();
    e->stile_idx.clear();
    e->res_reps.clear();
    int t = 0;
    DevBatch& d = e->d;
    for (int cls = 0; cls < 3; ++cls) {
        d.vclass_begin[cls] = t;
        d.vclass_width[cls] = widths[cls];
        for (SampleDesc& sd : e->samples) {
            if (sd.vec != widths[cls]) continue;
            sd.tile0 = t;
            const int nrep = e->C * sd.NT;
            for (int q = 0; q < nrep; ++q)
                for (int k = 0; k < sd.tiles_per_rep; ++k) {
                    e->tiles.push_back(make_int2(sd.r0 + q, k * TILE * sd.vec));
                    ++t;
                }
        }
        d.vclass_count[cls] = t - d.vclass_begin[cls];
    }
    for (int cls = 0; cls < 3; ++cls) {
        d.sclass_begin[cls] = (int)e->stile_idx.size();
        for (const SampleDesc& sd : e->samples) {
            if (sd.vec != widths[cls] || sd.resident) continue;
            const int n = e->C * sd.NT * sd.tiles_per_rep;
            for (int q = 0; q < n; ++q) e->stile_idx.push_back(sd.tile0 + q);
        }
        d.sclass_count[cls] = (int)e->stile_idx.size() - d.sclass_begin[cls];
    }
    e->any_streaming = false;
    for (const SampleDesc& sd : e->samples)
        if (!sd.resident) e->any_streaming = true;
    // resident replicas grouped by path (one CTA; wide or narrow clusters of
    // 2, 4, 8 CTAs)
    for (int g = 0; g < RES_GROUPS; ++g) {
        d.rcl_begin[g] = (int)e->res_reps.size();
        d.rcl_half[g] = 0;
        for (const SampleDesc& sd : e->samples) {
            if (!sd.resident || resident_group(sd.resident, sd.narrow != 0) != g) continue;
            for (int q = 0; q < e->C * sd.NT; ++q) e->res_reps.push_back(sd.r0 + q);
            d.rcl_half[g] = std::max(d.rcl_half[g], sd.half);
        }
        d.rcl_count[g] = (int)e->res_reps.size() - d.rcl_begin[g];
    }
    d.res_max_half = d.rcl_half[0];
    if ((size_t)t > e->tile_cap) return fail(PT_ERR_STATE, "tile list exceeds its capacity");
    // every sample streaming: the subset is the whole list, index it directly
    d.stiles = e->res_reps.empty() ? nullptr : e->d_stiles;
    e->T = t;
    d.n_tiles = t;
    d.n_res_reps = (int)e->res_reps.size();
    if (!e->tiles.empty())
        CK(cudaMemcpyAsync((void*)d.vtiles, e->tiles.data(), sizeof(int2) * e->tiles.size(), cudaMemcpyHostToDevice,
                           e->stream));
    if (!e->stile_idx.empty())
        CK(cudaMemcpyAsync(e->d_stiles, e->stile_idx.data(), sizeof(int) * e->stile_idx.size(),
                           cudaMemcpyHostToDevice, e->stream));
    if (!e->res_reps.empty())
        CK(cudaMemcpyAsync(e->d_res_reps, e->res_reps.data(), sizeof(int) * e->res_reps.size(),
                           cudaMemcpyHostToDevice, e->stream));
    CK(cudaMemcpyAsync((void*)d.samples, e->samples.data(), sizeof(SampleDesc) * e->samples.size(),
                       cudaMemcpyHostToDevice, e->stream));
    CK(e->stream ? cudaStreamSynchronize(e->stream) : cudaDeviceSynchronize());
    return PT_OK;
}

pt_status create_impl(pt_handle* out, int n_samples, const int* Ls, const int* NTs,
                      const float* const* Js, const double* const* betas, const pt_options* optp) {
    if (!out) return fail(PT_ERR_ARG, "out is NULL");
    *out = nullptr;
    pt_options opt;
    pt_options_default(&opt);
    if (optp) opt = *optp;
    if (n_samples < 1) return fail(PT_ERR_ARG, "n_samples must be >= 1 (got %d)", n_samples);
    if (opt.n_copies != 1 && opt.n_copies != 2) return fail(PT_ERR_ARG, "n_copies must be 1 or 2");
    if (opt.precision != PT_FP32 && opt.precision != PT_FP64) return fail(PT_ERR_ARG, "bad precision");
    if (opt.start != PT_START_RANDOM && opt.start != PT_START_ORDERED) return fail(PT_ERR_ARG, "bad start");
    if ((opt.alloc == nullptr) != (opt.free == nullptr)) return fail(PT_ERR_ARG, "alloc and free must be given together");
    if (!Ls || !NTs || !Js || !betas) return fail(PT_ERR_ARG, "NULL per-sample array");
    for (int s = 0; s < n_samples; ++s) {
        const int L = Ls[s];
        if (L < 2 || (L & 1)) return fail(PT_ERR_ODD_L, "sample %d: L = %d must be even and >= 2", s, L);
        if (L > 1024 || (long long)L * L * L >= (1LL << 30)) return fail(PT_ERR_ARG, "sample %d: L = %d too large", s, L);
        if (NTs[s] < 2 || NTs[s] > kMaxNT) return fail(PT_ERR_ARG, "sample %d: n_replicas = %d outside [2, %d]", s, NTs[s], kMaxNT);
        if (!Js[s] || !betas[s]) return fail(PT_ERR_ARG, "sample %d: NULL couplings or betas", s);
        for (int b = 0; b < NTs[s]; ++b) {
            const double v = betas[s][b];
            if (!std::isfinite(v) || v < 0.0) return fail(PT_ERR_ARG, "sample %d: beta[%d] = %g invalid", s, b, v);
            if (b > 0 && !(v > betas[s][b - 1])) return fail(PT_ERR_ARG, "sample %d: betas not strictly increasing at %d", s, b);
        }
        const long long n3 = 3LL * L * L * L;
        for (long long n = 0; n < n3; ++n)
            if (!std::isfinite(Js[s][n])) return fail(PT_ERR_ARG, "sample %d: coupling %lld not finite", s, n);
    }

    pt_engine* e = new (std::nothrow) pt_engine();
    if (!e) return fail(PT_ERR_NOMEM, "host allocation failed");
    e->S = n_samples;
    e->C = opt.n_copies;
    e->fp64 = opt.precision == PT_FP64;
    e->seed = opt.seed;
    e->start = opt.start;
    e->stream = (cudaStream_t)opt.stream;
    e->alloc = opt.alloc;
    e->freefn = opt.free;
    e->actx = opt.alloc_ctx;
    e->L.assign(Ls, Ls + n_samples);
    e->NT.assign(NTs, NTs + n_samples);

    // ---- descriptors ------------------------------------------------------
    long long J_off = 0, pool = 0;
    int beta_off = 0, eps_off = 0, r = 0, t = 0, pair = 0;
    std::vector<float> Jsplit;
    std::vector<double> beta_all;
    for (int s = 0; s < n_samples; ++s) {
        const int L = Ls[s], NT = NTs[s], N = L * L * L, half = N / 2, hL = L / 2;
        SampleDesc sd{};
        sd.L = L; sd.hL = hL; sd.half = half; sd.NT = NT;
        sd.div_hL = make_fastdiv((uint32_t)hL);
        sd.div_L = make_fastdiv((uint32_t)L);
        sd.J_off = J_off;
        sd.beta_off = beta_off;
        sd.eps_off = eps_off;
        sd.chain0 = (int)e->chains.size();
        sd.r0 = r;
        sd.vec = vec_width(hL, e->fp64);
        sd.tiles_per_rep = (half + TILE * sd.vec - 1) / (TILE * sd.vec);
        sd.tile0 = 0;  // set below, once tiles are grouped by class
        // colour-split forward couplings and the invertibility bound
        Jsplit.resize((size_t)(J_off + 3LL * N));
        const float* J = Js[s];
        float mx = 0.f;
        for (int x = 0; x < N; ++x) {
            const int i = x % L, j = (x / L) % L, k = x / (L * L);
            const int c = (i + j + k) & 1;
            const int h = (i >> 1) + hL * (j + L * k);
            const int xm[3] = {((i + L - 1) % L) + L * (j + L * k), i + L * (((j + L - 1) % L) + L * k),
                               i + L * (j + L * ((k + L - 1) % L))};
            float sum = 0.f;
            for (int mu = 0; mu < 3; ++mu) {
                Jsplit[(size_t)J_off + (size_t)c * 3 * half + (size_t)mu * half + h] = J[(size_t)mu * N + x];
                sum += std::fabs(J[(size_t)mu * N + x]) + std::fabs(J[(size_t)mu * N + xm[mu]]);
            }
            mx = std::max(mx, sum);
        }
        e->maxsumJ.push_back(mx);
        for (int b = 0; b < NT; ++b) {
            beta_all.push_back(betas[s][b]);
            e->q_sample.push_back(s);
        }
        for (int c = 0; c < e->C; ++c) {
            const int ch = (int)e->chains.size();
            e->chains.push_back(ChainDesc{s, c, r, pair});
            e->chain_off.push_back(pool);
            pool += (long long)(NT + 2) * 3 * N;
            for (int b = 0; b < NT; ++b) {
                e->reps.push_back(make_int4(s, ch, b, c * NT + b));
                ++r;
            }
            pair += NT - 1;
        }
        e->samples.push_back(sd);
        J_off += 3LL * N;
        beta_off += NT;
        eps_off += NT - 1;
    }
    // capacity of the tile lists: every sample at one site per thread
    for (const SampleDesc& sd : e->samples) e->tile_cap += (size_t)e->C * sd.NT * ((sd.half + TILE - 1) / TILE);
    // bulk-copy (TMA) half sweep: items of P planes x up to 16 replicas
    {
        // PT_TMA=1 selects the bulk-copy overrelaxation half sweep (opt-in:
        // measured slower than the vector-load kernel so far)
        const char* ev = std::getenv("PT_TMA");
        const bool allow = ev && std::strcmp(ev, "1") == 0;
        e->all_tma = allow;
        size_t smem = 0;
        for (SampleDesc& sd : e->samples) {
            sd.tma_planes = (!e->fp64 && sd.L % 8 == 0) ? tma_planes_for(sd.L) : 0;
            e->all_tma = e->all_tma && sd.tma_planes > 0;
            if (sd.tma_planes > 0) smem = std::max(smem, tma_smem_bytes(sd.tma_planes, sd.hL * sd.L));
        }
        if (smem > 220 * 1024) e->all_tma = false;
        if (e->all_tma) {
            for (const SampleDesc& sd : e->samples) {
                const int nrep = e->C * sd.NT;
                for (int k0 = 0; k0 < sd.L; k0 += sd.tma_planes)
                    for (int g = 0; g < nrep; g += 16)
                        e->tma_items.push_back(make_int4((int)(&sd - e->samples.data()), k0, sd.r0 + g,
                                                         std::min(16, nrep - g)));
            }
            e->d.tma_smem = (int)smem;
        }
    }
    for (const SampleDesc& sd : e->samples) e->max_half = std::max(e->max_half, sd.half);
    {
        // PT_CL_NARROW=1 prefers clusters of 512-thread CTAs (two per SM) for
        // samples too large for one CTA, until pt_autotune decides
        const char* ev = std::getenv("PT_CL_NARROW");
        e->narrow_default = ev && std::strcmp(ev, "1") == 0;
    }
    choose_paths(e);
    e->R = r;
    e->T = 0;
    e->P = pair;
    e->sumNT = beta_off;
    e->sumEps = eps_off;
    e->pool_elems = (size_t)pool;
    e->J_elems = (size_t)J_off;
    e->eps_host.assign((size_t)eps_off, 0.f);

    // ---- device memory ----------------------------------------------------
    pt_status st;
    DevBatch& d = e->d;
#define TRY(x)                   \
    do {                         \
        st = (x);                \
        if (st != PT_OK) {       \
            e->release();        \
            delete e;            \
            return st;           \
        }                        \
    } while (0)
    TRY(e->dalloc(&d.spins, e->pool_elems * e->esz()));
    float* dJ; TRY(upload(e, &dJ, Jsplit)); d.J = dJ;
    double* dB; TRY(upload(e, &dB, beta_all)); d.betas = dB;
    float* dE; TRY(upload(e, &dE, e->eps_host)); d.eps = dE;
    std::vector<int> ident(r), zero_i(r, 0), rts(r, 0);
    for (int q = 0; q < r; ++q) {
        ident[q] = e->reps[q].z;
        rts[q] = (e->reps[q].z == 0) ? 1 : 0;  // label 0 starts at b = 0
    }
    TRY(upload(e, &d.bufmap, ident));
    TRY(upload(e, &d.label, ident));
    TRY(upload(e, &d.rt_state, rts));
    std::vector<long long> zc((size_t)e->chains.size(), 0), zp((size_t)pair, 0);
    TRY(upload(e, &d.rt_count, zc));
    TRY(upload(e, &d.prop, zp));
    TRY(upload(e, &d.acc, zp));
    std::vector<double> zH((size_t)r, 0.0);
    TRY(upload(e, &d.H, zH));
    std::vector<int2> fb;
    for (size_t c = 0; c < e->chains.size(); ++c) {
        const int NT = e->NT[e->chains[c].s];
        fb.push_back(make_int2(NT, NT + 1));
    }
    TRY(upload(e, &d.freebuf, fb));
    SampleDesc* dS; TRY(upload(e, &dS, e->samples)); d.samples = dS;
    ChainDesc* dC; TRY(upload(e, &dC, e->chains)); d.chains = dC;
    int4* dR; TRY(upload(e, &dR, e->reps)); d.reps = dR;
    {
        std::vector<int2> zt2(e->tile_cap, make_int2(0, 0));
        std::vector<int> zti(e->tile_cap, 0), zr((size_t)r, 0), zn((size_t)n_samples, 0);
        int2* dT; TRY(upload(e, &dT, zt2)); d.vtiles = dT;
        TRY(upload(e, &e->d_stiles, zti)); d.stiles = e->d_stiles;
        TRY(upload(e, &e->d_res_reps, zr)); d.res_reps = e->d_res_reps;
        TRY(upload(e, &e->d_nor, zn));
        d.nor_s = nullptr;
    }
    int* dQs; TRY(upload(e, &dQs, e->q_sample)); d.q_sample = dQs;
    long long* dO; TRY(upload(e, &dO, e->chain_off)); d.chain_off = dO;
    std::vector<unsigned long long> z1(1, 0ull);
    TRY(upload(e, &d.d_step, z1));
    std::vector<int> zerr(1, 0);
    TRY(upload(e, &d.err, zerr));
    d.wait_limit = WAIT_LIMIT_DEFAULT;
    d.wait_fault = 0;
    int4* dTI; TRY(upload(e, &dTI, e->tma_items)); d.tma_items = dTI;
    d.n_tma_items = (int)e->tma_items.size();
    std::vector<double> zt(e->tile_cap, 0.0), zq((size_t)e->sumNT * 9, 0.0), zx((size_t)e->sumNT, 0.0);
    TRY(upload(e, &d.part, zt));
    TRY(upload(e, &d.Q, zq));
    TRY(upload(e, &d.chi, zx));
    std::vector<double> zl((size_t)pair * 3, 0.0);
    TRY(upload(e, &d.xlog, zl));
    std::vector<double> zd((size_t)pair * 2, 0.0);
    TRY(upload(e, &d.decim_pre, zd));
#undef TRY
    d.seed = e->seed;
    d.n_samples = e->S;
    d.n_chains = (int)e->chains.size();
    d.n_reps = r;
    d.n_q = e->sumNT;
    d.max_NT = 0;
    for (int v : e->NT) d.max_NT = std::max(d.max_NT, v);
    d.min_half = 1 << 30;
    for (const SampleDesc& sd : e->samples) d.min_half = std::min(d.min_half, sd.half);
    {
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
            d.n_sm = nsm;
        else
            d.n_sm = 1;
        // PT_EXCHANGE_CLUSTER = 1, 2, 4 or 8 fixes the CTAs per chain of the
        // decimation and cooling/heating exchanges (default: chosen from the
        // number of chains and SMs)
        const char* ev = std::getenv("PT_EXCHANGE_CLUSTER");
        const int cs = ev ? std::atoi(ev) : 0;
        d.exchange_cluster = (cs == 1 || cs == 2 || cs == 4 || cs == 8) ? cs : 0;
        // PT_EXCHANGE_IMPL = l2 | smem selects the exchange kernels (default:
        // shared-memory staged where the pair fits on one SM)
        const char* ei = std::getenv("PT_EXCHANGE_IMPL");
        d.exchange_impl = (ei && std::strcmp(ei, "l2") == 0) ? 1 : (ei && std::strcmp(ei, "smem") == 0) ? 2 : 0;
    }
    d.max_half = 0;
    for (const SampleDesc& sd : e->samples) d.max_half = std::max(d.max_half, sd.half);
    // the staged cooling/heating exchange keeps the heated proposal of every
    // pair (one configuration each) from the heating pre-pass through the walk
    // to the commit of the accepted ones
    d.heat_buf = nullptr;
    d.heat_H = d.heat_lnJ = nullptr;
    d.heat_commit = nullptr;
    if (exchange_smem_supported(2, d.max_half, e->fp64) && e->P > 0) {
        const size_t n = (size_t)e->P * 6 * (size_t)d.max_half;
        st = e->dalloc(&d.heat_buf, n * e->esz());
        if (st == PT_OK) st = e->dalloc((void**)&d.heat_H, sizeof(double) * (size_t)e->P);
        if (st == PT_OK) st = e->dalloc((void**)&d.heat_lnJ, sizeof(double) * (size_t)e->P);
        if (st == PT_OK) st = e->dalloc((void**)&d.heat_commit, sizeof(int) * (size_t)e->P);
        if (st != PT_OK) {
            e->release();
            delete e;
            return st;
        }
    }

    st = rebuild_lists(e);
    if (st == PT_OK)
        st = run(e, PT_KERNEL_OTHER, 1, [&]() { return launch_init_spins(d, e->fp64, e->start, e->stream); });
    if (st == PT_OK) st = compute_energy(e);
    if (st == PT_OK) {
        cudaError_t ce = e->stream ? cudaStreamSynchronize(e->stream) : cudaDeviceSynchronize();
        if (ce != cudaSuccess) st = fail(PT_ERR_CUDA, "create: %s", cudaGetErrorString(ce));
    }
    if (st != PT_OK) {
        e->release();
        delete e;
        return st;
    }
    *out = e;
    return PT_OK;
}

// Synchronise the engine's stream; report a bounded device-side wait that
// gave up since the last check (the error word is cleared).
pt_status sync(pt_engine* e) {
    // the error word rides on the stream behind the work, so one wait covers both
    if (!e->err_host) CK(cudaMallocHost((void**)&e->err_host, sizeof(int)));
    CK(cudaMemcpyAsync(e->err_host, e->d.err, sizeof(int), cudaMemcpyDeviceToHost, e->stream));
    CK(e->stream ? cudaStreamSynchronize(e->stream) : cudaDeviceSynchronize());
    const int err = *e->err_host;
    if (err) {
        const int zero = 0;
        CK(cudaMemcpy(e->d.err, &zero, sizeof(int), cudaMemcpyHostToDevice));
        return fail(PT_ERR_TIMEOUT, "a bounded device-side wait gave up (error word %d)", err);
    }
    return PT_OK;
}

pt_status check_eps(pt_engine* e, const float* eps) {
    for (int s = 0; s < e->S; ++s) {
        const SampleDesc& sd = e->samples[s];
        for (int i = 0; i < sd.NT - 1; ++i) {
            const float v = eps[sd.eps_off + i];
            if (!std::isfinite(v) || v < 0.f) return fail(PT_ERR_EPS, "sample %d pair %d: eps = %g invalid", s, i, v);
            if ((double)v * (double)e->maxsumJ[s] >= 1.0)
                return fail(PT_ERR_EPS, "sample %d pair %d: eps * max sum|J| = %g >= 1 (step not invertible)", s, i,
                            (double)v * e->maxsumJ[s]);
        }
    }
    return PT_OK;
}

pt_status locate(pt_engine* e, int sample, int copy, int replica, size_t* elem_off, int* L) {
    if (sample < 0 || sample >= e->S) return fail(PT_ERR_ARG, "sample %d out of range", sample);
    if (copy < 0 || copy >= e->C) return fail(PT_ERR_ARG, "copy %d out of range", copy);
    const SampleDesc& sd = e->samples[sample];
    if (replica < 0 || replica >= sd.NT) return fail(PT_ERR_ARG, "replica %d out of range", replica);
    const int ch = sd.chain0 + copy;
    const int r = e->chains[ch].r0 + replica;
    int buf = 0;
    CK(cudaMemcpyAsync(&buf, e->d.bufmap + r, sizeof(int), cudaMemcpyDeviceToHost, e->stream));
    pt_status st = sync(e);
    if (st != PT_OK) return st;
    *elem_off = (size_t)e->chain_off[ch] + (size_t)buf * 6 * sd.half;
    *L = sd.L;
    return PT_OK;
}

}  // namespace

extern "C" {

void pt_options_default(pt_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof *opt);
    opt->n_samples = 1;
    opt->n_copies = 2;
    opt->precision = PT_FP32;
    opt->seed = 0;
    opt->start = PT_START_RANDOM;
}

pt_status pt_create(pt_handle* out, int L, const float* couplings, const double* betas, int n_replicas,
                    const pt_options* opt) {
    pt_options o;
    pt_options_default(&o);
    if (opt) o = *opt;
    if (!couplings || !betas) return fail(PT_ERR_ARG, "NULL couplings or betas");
    if (o.n_samples < 1) return fail(PT_ERR_ARG, "n_samples must be >= 1");
    const long long N = (long long)L * L * L;
    std::vector<int> Ls((size_t)o.n_samples, L), NTs((size_t)o.n_samples, n_replicas);
    std::vector<const float*> Js((size_t)o.n_samples);
    std::vector<const double*> Bs((size_t)o.n_samples);
    for (int s = 0; s < o.n_samples; ++s) {
        Js[s] = couplings + (size_t)s * 3 * (size_t)(N > 0 ? N : 0);
        Bs[s] = betas + (size_t)s * (size_t)(n_replicas > 0 ? n_replicas : 0);
    }
    return create_impl(out, o.n_samples, Ls.data(), NTs.data(), Js.data(), Bs.data(), &o);
}

pt_status pt_create_batch(pt_handle* out, int n_samples, const int* L, const int* n_replicas,
                          const float* const* couplings, const double* const* betas, const pt_options* opt) {
    return create_impl(out, n_samples, L, n_replicas, couplings, betas, opt);
}

// One block of local updates.  nor == NULL: n_or sweeps for every sample;
// else nor[s] sweeps for sample s (n_or = their maximum).  Heat-bath half
// sweeps take the step counters 0 .. 2 n_hb - 1, overrelaxation half sweeps
// the following ones, whatever path a sample takes; the counter advances by
// 2 (n_hb + n_or).
static pt_status sweep_impl(pt_engine* e, int n_hb, int n_or, const int* nor) {
    const int total = 2 * (n_hb + n_or);
    if (total == 0) return PT_OK;
    if (nor) {
        if (e->nor_host.size() != (size_t)e->S || std::memcmp(e->nor_host.data(), nor, sizeof(int) * e->S) != 0) {
            e->nor_host.assign(nor, nor + e->S);
            CK(cudaMemcpyAsync(e->d_nor, e->nor_host.data(), sizeof(int) * e->S, cudaMemcpyHostToDevice, e->stream));
            CK(e->stream ? cudaStreamSynchronize(e->stream) : cudaDeviceSynchronize());
        }
        e->d.nor_s = e->d_nor;
    } else {
        e->d.nor_s = nullptr;
    }
    const bool fuse = (nor == nullptr);  // per-sample counts: energies after the block
    if (!e->res_reps.empty())
        RUN(PT_KERNEL_RESIDENT, resident_launch_count(e->d), launch_resident(e->d, e->fp64, n_hb, n_or, e->stream));
    if (e->any_streaming) {
        const int nl = sweep_stream_launch_count(e->d);
        const bool tma = e->all_tma && e->res_reps.empty() && nor == nullptr;
        int k = 0;
        for (int hb = 0; hb < n_hb; ++hb)
            for (int c = 0; c < 2; ++c, ++k) {
                const bool last = fuse && (k == total - 1);
                RUN(PT_KERNEL_HB, nl, launch_halfsweep(e->d, e->fp64, 1, last, c, k, -1, e->stream));
            }
        for (int o = 0; o < n_or; ++o)
            for (int c = 0; c < 2; ++c, ++k) {
                const bool last = fuse && (k == total - 1);
                if (tma && !last)
                    RUN(PT_KERNEL_OR, 1, launch_or_tma(e->d, c, e->stream));
                else
                    RUN(PT_KERNEL_OR, nl, launch_halfsweep(e->d, e->fp64, 0, last, c, k, o, e->stream));
            }
        if (!fuse)
            RUN(PT_KERNEL_ENERGY, energy_launch_count(e->d, false), launch_energy(e->d, e->fp64, false, e->stream));
        RUN(PT_KERNEL_ENERGY, 1, launch_energy_finalize(e->d, false, e->stream));
    }
    RUN(PT_KERNEL_OTHER, 1, launch_advance_step(e->d, total, e->stream));
    e->step_host += (uint64_t)total;
    e->energy_valid = true;
    return PT_OK;
}

pt_status pt_sweep(pt_handle e, int n_hb, int n_or) {
    if (!e) return fail(PT_ERR_ARG, "NULL handle");
    if (n_hb < 0 || n_or < 0) return fail(PT_ERR_ARG, "n_hb, n_or must be >= 0");
    return sweep_impl(e, n_hb, n_or, nullptr);
}

pt_status pt_sweep_samples(pt_handle e, int n_hb, const int* n_or) {
    if (!e || !n_or) return fail(PT_ERR_ARG, "NULL argument");
    if (n_hb < 0) return fail(PT_ERR_ARG, "n_hb must be >= 0");
    int mx = 0;
    for (int s = 0; s < e->S; ++s) {
        if (n_or[s] < 0) return fail(PT_ERR_ARG, "n_or[%d] < 0", s);
        mx = std::max(mx, n_or[s]);
    }
    return sweep_impl(e, n_hb, mx, n_or);
}

static pt_status exchange_impl(pt_engine* e, pt_mode mode, const float* eps) {
    if (mode != PT_PLAIN && mode != PT_DECIMATION && mode != PT_COOLHEAT) return fail(PT_ERR_ARG, "bad mode %d", (int)mode);
    if (eps) {
        pt_status st = check_eps(e, eps);
        if (st != PT_OK) return st;
        std::memcpy(e->eps_host.data(), eps, sizeof(float) * e->eps_host.size());
        pt_status st2 = stage_copy(e, (void*)e->d.eps, eps, sizeof(float) * e->eps_host.size());
        if (st2 != PT_OK) return st2;
    } else if (mode == PT_COOLHEAT) {
        pt_status st = check_eps(e, e->eps_host.data());
        if (st != PT_OK) return st;
    }
    if (!e->energy_valid) {
        pt_status st = compute_energy(e);
        if (st != PT_OK) return st;
    }
    RUN(PT_KERNEL_EXCHANGE, exchange_launch_count(e->d, e->fp64, (int)mode),
        launch_exchange(e->d, e->fp64, (int)mode, e->stream));
    RUN(PT_KERNEL_OTHER, 1, launch_advance_step(e->d, 1, e->stream));
    e->step_host += 1;
    return PT_OK;
}
pt_status pt_exchange(pt_handle e, pt_mode mode, const float* eps) {
    if (!e) return fail(PT_ERR_ARG, "NULL handle");
    return exchange_impl(e, mode, eps);
}

// n_cycles update cycles (sweep block, tempering update, and with `measure`
// the overlap reduction), as one captured CUDA graph replayed n_cycles times
// when the engine has its own stream and no per-kernel profiling is on; the
// graph is captured again whenever the arguments or the kernel paths change.
pt_status pt_cycles(pt_handle e, int n_cycles, int n_hb, int n_or, const int* n_or_samples, pt_mode mode,
                    int measure) {
    if (!e) return fail(PT_ERR_ARG, "NULL handle");
    if (n_cycles < 0 || n_hb < 0 || n_or < 0) return fail(PT_ERR_ARG, "negative count");
    if (mode != PT_PLAIN && mode != PT_DECIMATION && mode != PT_COOLHEAT) return fail(PT_ERR_ARG, "bad mode %d", (int)mode);
    if (measure && e->C != 2) return fail(PT_ERR_STATE, "overlap needs n_copies == 2");
    if (n_cycles == 0) return PT_OK;
    int mx = n_or;
    if (n_or_samples) {
        mx = 0;
        for (int s = 0; s < e->S; ++s) {
            if (n_or_samples[s] < 0) return fail(PT_ERR_ARG, "n_or_samples[%d] < 0", s);
            mx = std::max(mx, n_or_samples[s]);
        }
    }
    if (mode == PT_COOLHEAT) {
        pt_status st = check_eps(e, e->eps_host.data());
        if (st != PT_OK) return st;
    }
    if (!e->energy_valid) {
        pt_status st = compute_energy(e);
        if (st != PT_OK) return st;
    }
    auto one_cycle = [&]() -> pt_status {
        pt_status st = sweep_impl(e, n_hb, mx, n_or_samples);
        if (st == PT_OK) st = exchange_impl(e, mode, nullptr);
        if (st == PT_OK && measure) st = run(e, PT_KERNEL_MEASURE, 1, [&]() { return launch_overlap(e->d, e->fp64, e->stream); });
        return st;
    };
    if (!e->stream || e->profiling) {
        for (int c = 0; c < n_cycles; ++c) {
            pt_status st = one_cycle();
            if (st != PT_OK) return st;
        }
        return PT_OK;
    }
    if (n_or_samples &&
        (e->nor_host.size() != (size_t)e->S || std::memcmp(e->nor_host.data(), n_or_samples, sizeof(int) * e->S) != 0)) {
        e->nor_host.assign(n_or_samples, n_or_samples + e->S);
        CK(cudaMemcpyAsync(e->d_nor, e->nor_host.data(), sizeof(int) * e->S, cudaMemcpyHostToDevice, e->stream));
        CK(cudaStreamSynchronize(e->stream));
    }
    std::vector<long long> key = {n_hb, mx, n_or_samples ? 1 : 0, (long long)mode, measure, e->policy, e->T,
                                  (long long)e->res_reps.size(), (long long)e->d.wait_limit, e->d.wait_fault};
    if (n_or_samples) key.insert(key.end(), n_or_samples, n_or_samples + e->S);
    if (!e->graph_exec || key != e->graph_key) {
        if (e->graph_exec) cudaGraphExecDestroy(e->graph_exec);
        if (e->graph) cudaGraphDestroy(e->graph);
        e->graph_exec = nullptr;
        e->graph = nullptr;
        long long before[PT_KERNEL_KINDS];
        std::memcpy(before, e->launches, sizeof before);
        const uint64_t step_before = e->step_host;
        CK(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeRelaxed));
        pt_status st = one_cycle();
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamEndCapture(e->stream, &g);
        if (st != PT_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (ce != cudaSuccess) return fail(PT_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
        e->graph = g;
        CK(cudaGraphInstantiate(&e->graph_exec, g, 0));
        for (int k = 0; k < PT_KERNEL_KINDS; ++k) {
            e->graph_launches[k] = e->launches[k] - before[k];
            e->launches[k] = before[k];
        }
        e->graph_steps = (int)(e->step_host - step_before);
        e->step_host = step_before;
        e->graph_key = key;
    }
    for (int c = 0; c < n_cycles; ++c) {
        CK(cudaGraphLaunch(e->graph_exec, e->stream));
        for (int k = 0; k < PT_KERNEL_KINDS; ++k) e->launches[k] += e->graph_launches[k];
        e->step_host += (uint64_t)e->graph_steps;
    }
    e->energy_valid = true;
    return PT_OK;
}

// Time the candidate paths (resident / streaming) and vector widths of every
// lattice size of the batch on the batch itself and keep the fastest; the
// chain state (spins, energies, step counter) is restored afterwards.
pt_status pt_autotune(pt_handle e, int n_hb, int n_or, int* choice, double* best_ms) {
    if (!e) return fail(PT_ERR_ARG, "NULL handle");
    if (n_hb < 0 || n_or < 0 || n_hb + n_or == 0) return fail(PT_ERR_ARG, "need a positive sweep count");
    pt_status st = sync(e);
    if (st != PT_OK) return st;
    const bool saved_prof = e->profiling;
    e->profiling = false;
    void* backup = nullptr;
    const size_t pool_bytes = e->pool_elems * e->esz();
    cudaError_t ce = cudaMalloc(&backup, pool_bytes + sizeof(double) * e->R);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        e->profiling = saved_prof;
        return fail(PT_ERR_NOMEM, "autotune backup: %s", cudaGetErrorString(ce));
    }
    const uint64_t step0 = e->step_host;
    const bool ev0 = e->energy_valid;
    CK(cudaMemcpyAsync(backup, e->d.spins, pool_bytes, cudaMemcpyDeviceToDevice, e->stream));
    CK(cudaMemcpyAsync((char*)backup + pool_bytes, e->d.H, sizeof(double) * e->R, cudaMemcpyDeviceToDevice, e->stream));
    const int saved_policy = e->policy;
    e->policy = PT_POLICY_AUTO;
    e->tuned_vec.assign(e->S, 0);
    e->tuned_res.assign(e->S, -1);
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    std::vector<int> Ls;
    for (const SampleDesc& sd : e->samples)
        if (std::find(Ls.begin(), Ls.end(), sd.L) == Ls.end()) Ls.push_back(sd.L);
    std::vector<double> best(e->S, 0.0);
    for (int L : Ls) {
        const int hL = L / 2;
        std::vector<std::pair<int, int>> cand;  // (resident, vec)
        for (int res = 2; res >= 0; --res)
            for (int vec : {4, 2, 1}) {
                if (e->fp64 && vec == 4) continue;
                if (hL % vec) continue;
                if (res) {
                    bool ok = true;
                    for (const SampleDesc& sd : e->samples)
                        if (sd.L == L && (res == 2 ? resident_cluster_narrow(sd, e->fp64, vec)
                                                   : resident_cluster(sd, e->fp64, vec)) == 0)
                            ok = false;
                    if (!ok) continue;
                }
                cand.push_back({res, vec});
            }
        double best_t = 1e30;
        std::pair<int, int> best_c = cand.empty() ? std::make_pair(0, 1) : cand[0];
        for (auto c : cand) {
            for (int s = 0; s < e->S; ++s)
                if (e->samples[s].L == L) {
                    e->tuned_res[s] = c.first;
                    e->tuned_vec[s] = c.second;
                }
            choose_paths(e);
            st = rebuild_lists(e);
            if (st == PT_OK) st = sweep_impl(e, n_hb, n_or, nullptr);  // warm-up
            if (st != PT_OK) break;
            CK(cudaEventRecord(a, e->stream));
            for (int rep = 0; rep < 2 && st == PT_OK; ++rep) st = sweep_impl(e, n_hb, n_or, nullptr);
            CK(cudaEventRecord(b, e->stream));
            CK(cudaEventSynchronize(b));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, a, b));
            if (ms < best_t) {
                best_t = ms;
                best_c = c;
            }
        }
        if (st != PT_OK) break;
        for (int s = 0; s < e->S; ++s)
            if (e->samples[s].L == L) {
                e->tuned_res[s] = best_c.first;
                e->tuned_vec[s] = best_c.second;
                best[s] = best_t / 2;
            }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st == PT_OK) {
        choose_paths(e);
        st = rebuild_lists(e);
    }
    // restore the chain state
    cudaMemcpyAsync(e->d.spins, backup, pool_bytes, cudaMemcpyDeviceToDevice, e->stream);
    cudaMemcpyAsync(e->d.H, (char*)backup + pool_bytes, sizeof(double) * e->R, cudaMemcpyDeviceToDevice, e->stream);
    e->step_host = step0;
    cudaMemcpyAsync(e->d.d_step, &e->step_host, sizeof(uint64_t), cudaMemcpyHostToDevice, e->stream);
    cudaStreamSynchronize(e->stream);
    cudaFree(backup);
    e->energy_valid = ev0;
    e->profiling = saved_prof;
    if (saved_policy != PT_POLICY_AUTO) e->policy = PT_POLICY_AUTO;
    if (st != PT_OK) return st;
    for (int s = 0; s < e->S; ++s) {
        const SampleDesc& sd = e->samples[s];
        if (choice) choice[s] = sd.resident ? (sd.narrow ? 20 : 10) + sd.vec : sd.vec;
        if (best_ms) best_ms[s] = best[s];
    }
    return sync(e);
}

pt_status pt_measure(pt_handle e, double* energy, double* overlap, double* chi) {
    if (!e) return fail(PT_ERR_ARG, "NULL handle");
    if ((overlap || chi) && e->C != 2) return fail(PT_ERR_STATE, "overlap needs n_copies == 2");
    if (!e->energy_valid) {
        pt_status st = compute_energy(e);
        if (st != PT_OK) return st;
    }
    if (overlap || chi) RUN(PT_KERNEL_MEASURE, 1, launch_overlap(e->d, e->fp64, e->stream));
    if (energy) CK(cudaMemcpyAsync(energy, e->d.H, sizeof(double) * e->R, cudaMemcpyDeviceToHost, e->stream));
    if (overlap) CK(cudaMemcpyAsync(overlap, e->d.Q, sizeof(double) * 9 * e->sumNT, cudaMemcpyDeviceToHost, e->stream));
    if (chi) CK(cudaMemcpyAsync(chi, e->d.chi, sizeof(double) * e->sumNT, cudaMemcpyDeviceToHost, e->stream));
    return sync(e);
}

pt_status pt_measure_device(pt_handle e, double* d_energy, double* d_overlap, double* d_chi) {
    if (!e) return fail(PT_ERR_ARG, "NULL handle");
    if (e->C != 2 && (d_overlap || d_chi)) return fail(PT_ERR_STATE, "overlap needs n_copies == 2");
    if (!e->energy_valid) {
        pt_status st = compute_energy(e);
        if (st != PT_OK) return st;
    }
    if (e->C == 2) RUN(PT_KERNEL_MEASURE, 1, launch_overlap(e->d, e->fp64, e->stream));
    if (d_energy) CK(cudaMemcpyAsync(d_energy, e->d.H, sizeof(double) * e->R, cudaMemcpyDeviceToDevice, e->stream));
    if (d_overlap)
        CK(cudaMemcpyAsync(d_overlap, e->d.Q, sizeof(double) * 9 * e->sumNT, cudaMemcpyDeviceToDevice, e->stream));
    if (d_chi) CK(cudaMemcpyAsync(d_chi, e->d.chi, sizeof(double) * e->sumNT, cudaMemcpyDeviceToDevice, e->stream));
    return PT_OK;
}

pt_status pt_profile(pt_handle e, int enable) {
    if (!e) return fail(PT_ERR_ARG, "NULL handle");
    pt_status st = sync(e);
    if (st != PT_OK) return st;
    for (auto& r : e->recs) { e->ev_pool.push_back(r.a); e->ev_pool.push_back(r.b); }
    e->recs.clear();
    for (int k = 0; k < PT_KERNEL_KINDS; ++k) e->launches[k] = 0;
    e->profiling = enable != 0;
    return PT_OK;
}

pt_status pt_profile_read(pt_handle e, double* ms, int64_t* launches) {
    if (!e) return fail(PT_ERR_ARG, "NULL handle");
    pt_status st = sync(e);
    if (st != PT_OK) return st;
    double acc[PT_KERNEL_KINDS] = {0};
    for (auto& r : e->recs) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, r.a, r.b));
        acc[r.kind] += t;
    }
    for (int k = 0; k < PT_KERNEL_KINDS; ++k) {
        if (ms) ms[k] = acc[k];
        if (launches) launches[k] = e->launches[k];
    }
    return PT_OK;
}

pt_status pt_get_stats(pt_handle e, int64_t* proposals, int64_t* accepts, int64_t* round_trips, int32_t* perm) {
    if (!e) return fail(PT_ERR_ARG, "NULL handle");
    if (proposals) CK(cudaMemcpyAsync(proposals, e->d.prop, sizeof(int64_t) * e->P, cudaMemcpyDeviceToHost, e->stream));
    if (accepts) CK(cudaMemcpyAsync(accepts, e->d.acc, sizeof(int64_t) * e->P, cudaMemcpyDeviceToHost, e->stream));
    if (round_trips)
        CK(cudaMemcpyAsync(round_trips, e->d.rt_count, sizeof(int64_t) * e->chains.size(), cudaMemcpyDeviceToHost, e->stream));
    if (perm) CK(cudaMemcpyAsync(perm, e->d.label, sizeof(int32_t) * e->R, cudaMemcpyDeviceToHost, e->stream));
    return sync(e);
}

pt_status pt_get_exchange_log(pt_handle e, double* lnA, double* lnJ) {
    if (!e) return fail(PT_ERR_ARG, "NULL handle");
    if (!lnA && !lnJ) return PT_OK;
    std::vector<double> tmp((size_t)e->P * 3);
    CK(cudaMemcpyAsync(tmp.data(), e->d.xlog, sizeof(double) * tmp.size(), cudaMemcpyDeviceToHost, e->stream));
    const pt_status st = sync(e);
    if (st != PT_OK) return st;
    for (int q = 0; q < e->P; ++q) {
        if (lnA) lnA[q] = tmp[3 * (size_t)q];
        if (lnJ) {
            lnJ[2 * (size_t)q] = tmp[3 * (size_t)q + 1];
            lnJ[2 * (size_t)q + 1] = tmp[3 * (size_t)q + 2];
        }
    }
    return PT_OK;
}

pt_status pt_get_spins(pt_handle e, int sample, int copy, int replica, double* xyz) {
    if (!e || !xyz) return fail(PT_ERR_ARG, "NULL argument");
    size_t off;
    int L;
    pt_status st = locate(e, sample, copy, replica, &off, &L);
    if (st != PT_OK) return st;
    const size_t n = 3ull * L * L * L;
    std::vector<char> tmp(n * e->esz());
    CK(cudaMemcpyAsync(tmp.data(), (char*)e->d.spins + off * e->esz(), n * e->esz(), cudaMemcpyDeviceToHost, e->stream));
    st = sync(e);
    if (st != PT_OK) return st;
    if (e->fp64) split_to_natural(L, (const double*)tmp.data(), xyz);
    else split_to_natural(L, (const float*)tmp.data(), xyz);
    return PT_OK;
}

pt_status pt_set_spins(pt_handle e, int sample, int copy, int replica, const double* xyz) {
    if (!e || !xyz) return fail(PT_ERR_ARG, "NULL argument");
    size_t off;
    int L;
    pt_status st = locate(e, sample, copy, replica, &off, &L);
    if (st != PT_OK) return st;
    const size_t n = 3ull * L * L * L;
    for (size_t q = 0; q < n; ++q)
        if (!std::isfinite(xyz[q])) return fail(PT_ERR_ARG, "spin component %zu not finite", q);
    // unit vectors, as every update expects (its renormalisation corrects
    // rounding errors only): spins already unit to float accuracy are kept
    // as given, others are scaled to unit length
    std::vector<double> unit(xyz, xyz + n);
    for (size_t x = 0; x < n / 3; ++x) {
        double* v = &unit[3 * x];
        const double r2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        if (!(r2 > 0.0)) return fail(PT_ERR_ARG, "spin of site %zu is zero", x);
        if (std::fabs(r2 - 1.0) > 1e-6) {
            const double r = std::sqrt(r2);
            v[0] /= r; v[1] /= r; v[2] /= r;
        }
    }
    std::vector<char> tmp(n * e->esz());
    if (e->fp64) natural_to_split(L, unit.data(), (double*)tmp.data());
    else natural_to_split(L, unit.data(), (float*)tmp.data());
    CK(cudaMemcpyAsync((char*)e->d.spins + off * e->esz(), tmp.data(), n * e->esz(), cudaMemcpyHostToDevice, e->stream));
    e->energy_valid = false;
    return sync(e);
}

pt_status pt_set_params(pt_handle e, const double* betas, const float* eps) {
    if (!e) return fail(PT_ERR_ARG, "NULL handle");
    if (betas) {
        for (int s = 0; s < e->S; ++s) {
            const SampleDesc& sd = e->samples[s];
            for (int b = 0; b < sd.NT; ++b) {
                const double v = betas[sd.beta_off + b];
                if (!std::isfinite(v) || v < 0.0) return fail(PT_ERR_ARG, "sample %d: beta[%d] invalid", s, b);
                if (b > 0 && !(v > betas[sd.beta_off + b - 1])) return fail(PT_ERR_ARG, "sample %d: betas not increasing", s);
            }
        }
    }
    if (eps) {
        for (int q = 0; q < e->sumEps; ++q)
            if (!std::isfinite(eps[q]) || eps[q] < 0.f) return fail(PT_ERR_EPS, "eps[%d] invalid", q);
    }
    if (betas) {
        pt_status st = stage_copy(e, (void*)e->d.betas, betas, sizeof(double) * e->sumNT);
        if (st != PT_OK) return st;
    }
    if (eps) {
        std::memcpy(e->eps_host.data(), eps, sizeof(float) * e->eps_host.size());
        pt_status st = stage_copy(e, (void*)e->d.eps, eps, sizeof(float) * e->sumEps);
        if (st != PT_OK) return st;
    }
    return PT_OK;
}

pt_status pt_set_rng_step(pt_handle e, uint64_t step) {
    if (!e) return fail(PT_ERR_ARG, "NULL handle");
    e->step_host = step;
    CK(cudaMemcpyAsync(e->d.d_step, &e->step_host, sizeof(uint64_t), cudaMemcpyHostToDevice, e->stream));
    return sync(e);
}

pt_status pt_get_rng_step(pt_handle e, uint64_t* step) {
    if (!e || !step) return fail(PT_ERR_ARG, "NULL argument");
    unsigned long long v = 0;
    CK(cudaMemcpyAsync(&v, e->d.d_step, sizeof v, cudaMemcpyDeviceToHost, e->stream));
    pt_status st = sync(e);
    if (st != PT_OK) return st;
    *step = v;
    return PT_OK;
}

// Checkpoint file: magic, header of shapes, then the device arrays in a
// fixed order.
namespace {
struct CkptHeader {
    char magic[8];
    int version, S, C, fp64, R, P, T, sumNT, sumEps, n_chains, energy_valid;
    long long pool_elems;
    unsigned long long seed, step;
};

struct Blob {
    void* dev;
    size_t bytes;
};

std::vector<Blob> state_blobs(pt_engine* e) {
    return {{e->d.spins, e->pool_elems * e->esz()},
            {e->d.bufmap, sizeof(int) * e->R},
            {e->d.label, sizeof(int) * e->R},
            {e->d.rt_state, sizeof(int) * e->R},
            {e->d.rt_count, sizeof(long long) * e->chains.size()},
            {e->d.prop, sizeof(long long) * e->P},
            {e->d.acc, sizeof(long long) * e->P},
            {e->d.H, sizeof(double) * e->R},
            {e->d.freebuf, sizeof(int2) * e->chains.size()},
            {(void*)e->d.betas, sizeof(double) * e->sumNT},
            {(void*)e->d.eps, sizeof(float) * e->sumEps}};
}
}  // namespace

pt_status pt_save(pt_handle e, const char* path) {
    if (!e || !path) return fail(PT_ERR_ARG, "NULL argument");
    CkptHeader hd{};
    std::memcpy(hd.magic, "PTGB300", 8);
    hd.version = 1;
    hd.S = e->S; hd.C = e->C; hd.fp64 = e->fp64; hd.R = e->R; hd.P = e->P; hd.T = e->T;
    hd.sumNT = e->sumNT; hd.sumEps = e->sumEps; hd.n_chains = (int)e->chains.size();
    hd.energy_valid = e->energy_valid;
    hd.pool_elems = (long long)e->pool_elems;
    hd.seed = e->seed;
    unsigned long long step = 0;
    CK(cudaMemcpyAsync(&step, e->d.d_step, sizeof step, cudaMemcpyDeviceToHost, e->stream));
    pt_status st = sync(e);
    if (st != PT_OK) return st;
    hd.step = step;
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(PT_ERR_ARG, "cannot open %s for writing", path);
    bool ok = std::fwrite(&hd, sizeof hd, 1, f) == 1;
    for (const Blob& b : state_blobs(e)) {
        if (!ok) break;
        std::vector<char> tmp(b.bytes);
        cudaError_t ce = cudaMemcpy(tmp.data(), b.dev, b.bytes, cudaMemcpyDeviceToHost);
        if (ce != cudaSuccess) {
            std::fclose(f);
            return fail(PT_ERR_CUDA, "save: %s", cudaGetErrorString(ce));
        }
        ok = std::fwrite(tmp.data(), 1, b.bytes, f) == b.bytes;
    }
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(PT_ERR_ARG, "write to %s failed", path);
    return PT_OK;
}

pt_status pt_load(pt_handle e, const char* path) {
    if (!e || !path) return fail(PT_ERR_ARG, "NULL argument");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(PT_ERR_ARG, "cannot open %s", path);
    CkptHeader hd{};
    if (std::fread(&hd, sizeof hd, 1, f) != 1 || std::memcmp(hd.magic, "PTGB300", 8) != 0 || hd.version != 1) {
        std::fclose(f);
        return fail(PT_ERR_ARG, "%s is not a checkpoint of this engine", path);
    }
    if (hd.S != e->S || hd.C != e->C || hd.fp64 != (int)e->fp64 || hd.R != e->R || hd.P != e->P ||
        hd.sumNT != e->sumNT || hd.n_chains != (int)e->chains.size() || hd.pool_elems != (long long)e->pool_elems) {
        std::fclose(f);
        return fail(PT_ERR_STATE, "checkpoint shapes do not match the handle");
    }
    std::vector<std::vector<char>> data;
    for (const Blob& b : state_blobs(e)) {
        std::vector<char> tmp(b.bytes);
        if (std::fread(tmp.data(), 1, b.bytes, f) != b.bytes) {
            std::fclose(f);
            return fail(PT_ERR_ARG, "%s is truncated", path);
        }
        data.push_back(std::move(tmp));
    }
    std::fclose(f);
    pt_status st = sync(e);
    if (st != PT_OK) return st;
    size_t q = 0;
    for (const Blob& b : state_blobs(e)) {
        CK(cudaMemcpy(b.dev, data[q].data(), b.bytes, cudaMemcpyHostToDevice));
        ++q;
    }
    // host mirrors of the parameters
    std::memcpy(e->eps_host.data(), data.back().data(), sizeof(float) * e->sumEps);
    e->seed = hd.seed;
    e->d.seed = hd.seed;
    e->step_host = hd.step;
    CK(cudaMemcpy(e->d.d_step, &hd.step, sizeof hd.step, cudaMemcpyHostToDevice));
    e->energy_valid = hd.energy_valid != 0;
    return PT_OK;
}

pt_status pt_set_policy(pt_handle e, int policy) {
    if (!e) return fail(PT_ERR_ARG, "NULL handle");
    if (policy != PT_POLICY_AUTO && policy != PT_POLICY_STREAMING && policy != PT_POLICY_RESIDENT)
        return fail(PT_ERR_ARG, "bad policy %d", policy);
    if (policy == PT_POLICY_RESIDENT && !e->all_resident)
        return fail(PT_ERR_STATE, "a sample does not fit the resident sweep kernel");
    pt_status st = sync(e);
    if (st != PT_OK) return st;
    e->policy = policy;
    choose_paths(e);
    return rebuild_lists(e);
}

pt_status pt_set_wait_limit(pt_handle e, unsigned long long limit, int inject) {
    if (!e) return fail(PT_ERR_ARG, "NULL handle");
    if (inject && (!e->all_tma || e->tma_items.empty()) && e->res_reps.empty())
        return fail(PT_ERR_STATE, "the batch runs no bulk-copy kernel (neither resident sweeps nor the bulk-copy half sweep)");
    pt_status st = sync(e);
    if (st != PT_OK) return st;
    e->d.wait_limit = limit ? limit : WAIT_LIMIT_DEFAULT;
    e->d.wait_fault = inject ? 1 : 0;
    return PT_OK;
}

pt_status pt_get_paths(pt_handle e, int* choice, int* ctas) {
    if (!e || !choice) return fail(PT_ERR_ARG, "NULL argument");
    for (int s = 0; s < e->S; ++s) {
        const SampleDesc& sd = e->samples[s];
        choice[s] = sd.resident ? (sd.narrow ? 20 : 10) + sd.vec : sd.vec;
        if (ctas) ctas[s] = sd.resident;
    }
    return PT_OK;
}

pt_status pt_set_paths(pt_handle e, const int* choice) {
    if (!e || !choice) return fail(PT_ERR_ARG, "NULL argument");
    for (int s = 0; s < e->S; ++s) {
        const SampleDesc& sd = e->samples[s];
        const int res = choice[s] / 10, vec = choice[s] % 10;
        if (choice[s] < 0 || res > 2 || (vec != 1 && vec != 2 && vec != 4) || sd.hL % vec || (e->fp64 && vec == 4))
            return fail(PT_ERR_ARG, "sample %d: path code %d is not a path of this sample", s, choice[s]);
        if (res == 1 && resident_cluster(sd, e->fp64, vec) == 0)
            return fail(PT_ERR_STATE, "sample %d: no resident kernel with %d sites per thread", s, vec);
        if (res == 2 && resident_cluster_narrow(sd, e->fp64, vec) == 0)
            return fail(PT_ERR_STATE, "sample %d: no narrow cluster with %d sites per thread", s, vec);
    }
    pt_status st = sync(e);
    if (st != PT_OK) return st;
    e->tuned_vec.assign(e->S, 0);
    e->tuned_res.assign(e->S, -1);
    for (int s = 0; s < e->S; ++s) {
        e->tuned_vec[s] = choice[s] % 10;
        e->tuned_res[s] = choice[s] / 10;
    }
    e->policy = PT_POLICY_AUTO;
    choose_paths(e);
    return rebuild_lists(e);
}

pt_status pt_destroy(pt_handle e) {
    if (!e) return PT_OK;
    e->release();
    delete e;
    return PT_OK;
}

const char* pt_last_error(void) { return g_err; }

}  // extern "C"
