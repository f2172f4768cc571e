// kernels.h -- host-side launchers of the engine's CUDA kernels (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pt_types.h"

namespace ptk {

// Groups of resident replicas (see DevBatch::rcl_begin).
constexpr int RES_GROUPS = 7;

// Polls of a bounded mbarrier wait before it gives up (the default of
// DevBatch::wait_limit, and the least the drain after a failed wait uses).
constexpr unsigned long long WAIT_LIMIT_DEFAULT = 1ull << 22;

// Raise a kernel's dynamic shared-memory limit once per kernel, device and
// size (later launches of the same or a smaller size skip the call).
cudaError_t ensure_smem(const void* kernel, size_t bytes);

// Everything a kernel may need about the batch; pointers are device pointers.
struct DevBatch {
    void* spins;                    // float or double pool (see pt_types.h)
    const float* J;                 // colour-split forward couplings
    const double* betas;            // [sum NT]
    const float* eps;               // [sum (NT - 1)]
    int* bufmap;                    // [R] physical buffer of replica r
    int* label;                     // [R] identity of the configuration at r
    int* rt_state;                  // [R] round-trip state, indexed r0 + label
    long long* rt_count;            // [chains]
    long long* prop;                // [pairs]
    long long* acc;                 // [pairs]
    double* H;                      // [R] energy of the configuration at r
    int2* freebuf;                  // [chains] two scratch buffers
    const SampleDesc* samples;      // [S]
    const ChainDesc* chains;        // [chains]
    const int4* reps;               // [R] (sample, chain, b, copy*NT + b)
    const int2* vtiles;             // [T] (replica, first h) of the half-sweep tiles (all samples)
    const int* stiles;              // indices into vtiles of the streaming samples' tiles
    const int* res_reps;            // replicas of the resident samples
    const int* nor_s;               // per-sample overrelaxation sweeps of the current block (or NULL)
    int n_res_reps, res_max_half;
    const int* q_sample;            // [sum NT] sample of each (sample, beta) pair
    const long long* chain_off;     // [chains] element offset of buffer 0
    unsigned long long* d_step;     // Philox step counter
    unsigned long long seed;
    double* part;                   // [T] per-tile energy partials
    double* Q;                      // [sum NT][9]
    double* chi;                    // [sum NT]
    int n_samples, n_chains, n_reps, n_tiles, n_q;
    int max_NT;
    int min_half;                   // smallest L^3/2 of the batch
    int n_sm;                       // multiprocessors of the device
    int exchange_cluster;           // CTAs per chain in the exchange (0: automatic)
    int exchange_impl;              // 0 automatic, 1 global-memory clusters, 2 shared-memory staged
    int max_half;                   // largest L^3/2 of the batch
    int* err;                       // device error word (bit 0: a bounded wait gave up)
    unsigned long long wait_limit;  // polls of a bounded mbarrier wait before it gives up
    int wait_fault;                 // test hook: CTA 0 of a bulk-copy kernel leaves its copies un-issued
    const int4* tma_items;          // (sample, k0, first replica, count) of the bulk-copy half sweep
    int n_tma_items;
    int tma_smem;                   // dynamic shared memory of the bulk-copy half sweep
    // half-sweep tiles are grouped by vector width (sites per thread); the
    // streaming subset is grouped the same way inside stiles
    int vclass_begin[3], vclass_count[3], vclass_width[3];
    int sclass_begin[3], sclass_count[3];
    // resident replicas grouped by path: 0 one CTA per replica; 1, 2, 3
    // clusters of 2, 4, 8 CTAs of 1024 threads; 4, 5, 6 clusters of 2, 4, 8
    // CTAs of 512 threads (two per SM): slices of res_reps and the largest
    // L^3/2 of each group
    int rcl_begin[RES_GROUPS], rcl_count[RES_GROUPS], rcl_half[RES_GROUPS];
    // cooling/heating with the pair staged in shared memory: the heated
    // configuration of every pair (pair index x 6 max_half elements), its
    // energy and ln det J_C, computed before the pairs are walked (NULL when
    // that exchange is not available to the batch)
    void* heat_buf;
    double* heat_H;
    double* heat_lnJ;
    int* heat_commit;  // [pairs] buffer an accepted heated proposal goes to, -1 if rejected
    // [pairs][2] the decimation sums T1, T2 of every pair over the
    // configurations as the update found them (cluster decimation walk)
    double* decim_pre;
    // [pairs][3]: ln A, ln det J_C(s1), ln det J_C(C^-1 s2) of each pair's
    // most recent proposal (the two Jacobian terms are 0 for the standard
    // and decimation swaps)
    double* xlog;
};

// Record the text returned by pt_last_error() for the calling thread.
void set_last_error(const char* msg);

// Number of kernels one half sweep launches (one per vector-width class).
int sweep_launch_count(const DevBatch& b);

// Half sweeps of the streaming samples (kind 0 = overrelaxation, 1 = heat
// bath); `energy` also writes the per-tile energy partials of the updated
// colour (valid for colour 1).  or_index >= 0 skips samples whose per-sample
// overrelaxation count (nor_s) is <= or_index.
cudaError_t launch_halfsweep(const DevBatch& b, bool fp64, int kind, bool energy, int color,
                             int step_k, int or_index, cudaStream_t st);
int sweep_stream_launch_count(const DevBatch& b);
// Energy partials of every sample (all = true) or of the streaming samples.
cudaError_t launch_energy(const DevBatch& b, bool fp64, bool all, cudaStream_t st);
int energy_launch_count(const DevBatch& b, bool all);
// H[r] from the partials, for every replica (all) or the streaming samples'.
cudaError_t launch_energy_finalize(const DevBatch& b, bool all, cudaStream_t st);
cudaError_t launch_init_spins(const DevBatch& b, bool fp64, int ordered, cudaStream_t st);
cudaError_t launch_advance_step(const DevBatch& b, int by, cudaStream_t st);
cudaError_t launch_overlap(const DevBatch& b, bool fp64, cudaStream_t st);
cudaError_t launch_exchange(const DevBatch& b, bool fp64, int mode, cudaStream_t st);
// Kernels one tempering update launches.
int exchange_launch_count(const DevBatch& b, bool fp64, int mode);

// Decimation / cooling-heating exchanges with the pair staged in shared
// memory (one CTA per chain), for configurations that fit on one SM.
bool exchange_smem_supported(int mode, int max_half, bool fp64);
cudaError_t launch_exchange_smem(const DevBatch& b, bool fp64, int mode, int max_half, cudaStream_t st);

// Overrelaxation half sweep with the slab and halo staged by bulk copies
// (float, L % 8 == 0); tma_planes_for gives the planes per work item.
bool tma_supported(const SampleDesc& sd, bool fp64);
int tma_planes_for(int L);
size_t tma_smem_bytes(int P, int plane);
cudaError_t launch_or_tma(const DevBatch& b, int color, cudaStream_t st);

// Resident sweep blocks: one CTA per replica runs n_hb + n_or sweeps in shared
// memory and writes H[r].
bool resident_supported(const SampleDesc& sd, bool fp64, int vec);
// CTAs that hold one replica of the sample on chip: 1 when one CTA can
// (resident_supported), else the smallest cluster of 2, 4 or 8 CTAs that can
// (each CTA a slab of L/size z planes), 0 when none can.
int resident_cluster(const SampleDesc& sd, bool fp64, int vec);

// Narrow clusters: the smallest cluster of 2, 4 or 8 CTAs of 512 threads whose
// slab fits two CTAs per SM (<= 110 KB), for samples that do not fit one CTA;
// 0 if none.
int resident_cluster_narrow(const SampleDesc& sd, bool fp64, int vec);

// Group of a resident replica (DevBatch::rcl_begin) for cs CTAs per replica.
int resident_group(int cs, bool narrow);
// Kernels one resident block launches (one per non-empty group).
int resident_launch_count(const DevBatch& b);
cudaError_t launch_resident(const DevBatch& b, bool fp64, int n_hb, int n_or, cudaStream_t st);

}  // namespace ptk
