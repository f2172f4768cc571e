/*
 * pt.h -- C ABI of the GB300 parallel-tempering engine for the
 * three-dimensional Heisenberg Edwards-Anderson spin glass.
 *
 * Method: M. Hasenbusch and S. Schaefer, "Speeding up parallel tempering
 * simulations", arXiv:1006.4247.  N replicas of the model at inverse
 * temperatures beta_1 < ... < beta_N are updated independently (heat bath +
 * overrelaxation, section III.C) and configurations are exchanged between
 * neighbouring temperatures (section I, Eq. 1; improved exchanges of sections
 * III.A and III.B).  Observables are the energy and the overlap (section II).
 *
 * Model (section I): periodic L x L x L simple-cubic lattice, N = L^3 sites,
 * unit three-component spins s_x, H = - sum_<xy> J_xy s_x . s_y.
 *
 * Conventions used throughout this header
 *   site x = i + L*(j + L*k); colour c(x) = (i + j + k) mod 2 ("black" = 0);
 *   bond (x, mu) joins x and x + e_mu (periodic) and carries J[mu][x];
 *   a chain is (sample, copy); the two copies of a sample are independent
 *   Markov chains used for the overlap (section II);
 *   "replica" b (0 <= b < n_replicas) is the inverse-temperature index, betas
 *   strictly increasing with b;
 *   host arrays are C-contiguous and caller-owned; the library copies what it
 *   needs and never keeps a host pointer;
 *   device memory belongs to the handle (or to the allocator callback) and is
 *   released by pt_destroy.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), counter
 * based, no stored state:
 *   key = (seed_lo32, seed_hi32 XOR sample)
 *   ctr = (c0, c1, step_lo32, (purpose << 24) | (step_hi32 & 0xFFFFFF))
 *   purpose 0 heat bath (c0 = x, c1 = copy*n_replicas + b),
 *           1 exchange uniform (c0 = pair index, c1 = copy),
 *           2 decimation re-insertion (c0 = x, c1 = copy*n_replicas + b),
 *           3 decimation first colour (c0 = 0, c1 = copy),
 *           4 initial spins (c0 = x, c1 = copy*n_replicas + b, step 0).
 *   The step counter advances by one per half sweep (pt_sweep) and by one per
 *   pt_exchange call; it is shared by all chains.
 *
 * Errors: every call returns a pt_status and never aborts; pt_last_error()
 * describes the last failure of the calling thread.  A failed call leaves the
 * handle usable, except after PT_ERR_CUDA caused by a sticky CUDA error.
 *
 * Ordering: calls that only enqueue device work (pt_sweep, pt_exchange,
 * pt_set_params, pt_cycles, pt_measure_device) return before the work
 * completes; calls that return host
 * data (pt_measure, pt_get_stats, pt_get_spins, pt_save) synchronise the
 * engine's stream first.
 */
#ifndef PT_H
#define PT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pt_engine *pt_handle;

typedef enum {
    PT_OK = 0,
    PT_ERR_ARG = -1,      /* invalid argument (NULL, size, range, non-finite) */
    PT_ERR_ODD_L = -2,    /* L odd or < 2: the checkerboard needs a bipartite lattice */
    PT_ERR_EPS = -3,      /* cooling parameter makes the elementary step non-invertible */
    PT_ERR_CUDA = -4,     /* a CUDA call failed (text in pt_last_error) */
    PT_ERR_TIMEOUT = -5,  /* a bounded device-side wait gave up */
    PT_ERR_STATE = -6,    /* call not valid in the handle's state (e.g. overlap with 1 copy) */
    PT_ERR_NOMEM = -7     /* device or host allocation failed */
} pt_status;

typedef enum {
    PT_PLAIN = 0,       /* standard swap, section I Eq. 1 */
    PT_DECIMATION = 1,  /* decimation swap, section III.A Eq. aswap */
    PT_COOLHEAT = 2     /* cooling/heating swap, section III.B */
} pt_mode;

typedef enum { PT_FP32 = 0, PT_FP64 = 1 } pt_precision;
typedef enum { PT_START_RANDOM = 0, PT_START_ORDERED = 1 } pt_start;

/* Optional device allocator (for example a framework's caching allocator).
 * alloc returns a device pointer aligned to at least 256 bytes or NULL. */
typedef void *(*pt_alloc_fn)(size_t bytes, void *ctx);
typedef void (*pt_free_fn)(void *ptr, void *ctx);

typedef struct {
    int n_samples;        /* disorder samples (independent J sets), >= 1 */
    int n_copies;         /* 1 or 2 chains per sample (2 needed for the overlap) */
    int precision;        /* pt_precision of the spins and sweep arithmetic */
    uint64_t seed;        /* Philox seed */
    int start;            /* pt_start: uniform on the sphere, or all (1,0,0)
                             as in the equilibration study of section IV.C */
    void *stream;         /* cudaStream_t for all device work; NULL = legacy stream */
    pt_alloc_fn alloc;    /* NULL: cudaMalloc */
    pt_free_fn free;      /* NULL: cudaFree */
    void *alloc_ctx;
} pt_options;

/* Fill *opt with defaults: 1 sample, 2 copies, FP32, seed 0, random start,
 * NULL stream, cudaMalloc. */
void pt_options_default(pt_options *opt);

/* Create an engine for n_samples samples of one lattice size.
 *   L          even, >= 2 (PT_ERR_ODD_L otherwise)
 *   couplings  host float [n_samples][3][L^3], J[mu][x] of bond (x, x + e_mu);
 *              finite values (section I: Gaussian, zero mean, unit variance)
 *   betas      host double [n_samples][n_replicas], strictly increasing per
 *              sample, finite, >= 0
 *   n_replicas inverse temperatures per copy, >= 2
 * Spins start as opt->start says; the energies are computed; the
 * temperature-to-configuration map is the identity; counters are zero. */
pt_status pt_create(pt_handle *out, int L, const float *couplings,
                    const double *betas, int n_replicas, const pt_options *opt);

/* Create an engine for samples of different sizes in one batch.
 *   L[s], n_replicas[s]       per sample (same rules as pt_create)
 *   couplings[s]              host float [3][L[s]^3]
 *   betas[s]                  host double [n_replicas[s]]
 * opt->n_samples is ignored (n_samples is used).  Per-sample arrays returned
 * by the other calls are concatenated sample by sample (copy-major inside a
 * sample) instead of being rectangular. */
pt_status pt_create_batch(pt_handle *out, int n_samples, const int *L,
                          const int *n_replicas, const float *const *couplings,
                          const double *const *betas, const pt_options *opt);

/* Enqueue one block of local updates on every replica of every chain:
 * n_hb heat-bath sweeps, then n_or overrelaxation sweeps (section III.C; the
 * paper's cycle is 1 + 5L/4, section IV).  Each sweep is a colour-0 half sweep
 * followed by a colour-1 half sweep (checkerboard order).  n_hb, n_or >= 0. */
pt_status pt_sweep(pt_handle h, int n_hb, int n_or);

/* Like pt_sweep with a per-sample number of overrelaxation sweeps:
 * n_or[s] (host int [n_samples], >= 0) for sample s, e.g. the paper's 5L/4
 * in a batch of uneven L.  The step counter advances as for
 * pt_sweep(n_hb, max_s n_or[s]). */
pt_status pt_sweep_samples(pt_handle h, int n_hb, const int *n_or);

/* Enqueue one tempering update of every chain: pairs (b, b+1) for
 * b = 0 .. n_replicas-2 in increasing beta, one after the other.
 *   mode  PT_PLAIN: accept the swap with min[1, exp((b_{i+1}-b_i)(H_{i+1}-H_i))]
 *         PT_DECIMATION: swap one colour under the decimated action, the
 *           decimated colour alternating from pair to pair, the first one
 *           random; on acceptance re-insert the decimated colour by heat bath
 *         PT_COOLHEAT: propose the cooled configuration of beta_i at beta_{i+1}
 *           and the heated configuration of beta_{i+1} at beta_i
 *   eps   host float [n_samples][n_replicas-1] cooling parameters (copied and
 *         kept for later calls), or NULL to use the stored ones (default 0).
 *         PT_ERR_EPS if eps * max_x sum_{6 bonds} |J| >= 1 for any pair, or
 *         eps < 0. */
pt_status pt_exchange(pt_handle h, pt_mode mode, const float *eps);

/* Synchronise and copy observables to the host (each pointer may be NULL):
 *   energy  double [n_samples][n_copies][n_replicas]: H of the configuration
 *           at each beta (H = -sum J s.s; the paper's E is -H/L^3)
 *   overlap double [n_samples][n_replicas][9]: Q_ab = sum_x s^(0)_a,x s^(1)_b,x
 *           between the two copies at the same beta (section II)
 *   chi     double [n_samples][n_replicas]: chi = (1/L^3) sum_ab Q_ab^2
 * overlap/chi need n_copies == 2 (PT_ERR_STATE otherwise). */
pt_status pt_measure(pt_handle h, double *energy, double *overlap, double *chi);

/* Enqueue the same reductions as pt_measure without synchronising; results
 * are written to caller-owned DEVICE buffers of the same layouts (each may be
 * NULL, in which case the result is computed into the engine's own buffers
 * only).  For graph capture and for keeping time series on the device. */
pt_status pt_measure_device(pt_handle h, double *d_energy, double *d_overlap, double *d_chi);

/* Synchronise and copy the exchange bookkeeping (each pointer may be NULL):
 *   proposals, accepts  int64 [n_samples][n_copies][n_replicas-1] per pair
 *   round_trips         int64 [n_samples][n_copies]: completed trips
 *                       beta_0 -> beta_{N-1} -> beta_0 (section IV.B)
 *   perm                int32 [n_samples][n_copies][n_replicas]: identity
 *                       (initial replica index) of the configuration now at b */
pt_status pt_get_stats(pt_handle h, int64_t *proposals, int64_t *accepts,
                       int64_t *round_trips, int32_t *perm);

/* Synchronise and copy, per pair, the terms of the most recent tempering
 * update's proposal (each pointer may be NULL):
 *   lnA  double [n_samples][n_copies][n_replicas-1]: the log acceptance ratio
 *        the Metropolis test used (section I Eq. 1; section III.A Eq. aswap;
 *        section III.B, ln A = -b2 H[C s1] - b1 H[C^-1 s2] + b1 H[s1]
 *        + b2 H[s2] + ln det J_C(s1) - ln det J_C(C^-1 s2))
 *   lnJ  double [n_samples][n_copies][n_replicas-1][2]: for cooling/heating
 *        ln det J_C(s1) and ln det J_C(C^-1 s2) of that proposal (the
 *        Jacobian of the cooling sweep at the configuration it cools, and at
 *        the pre-image of the heated one); 0 for the other exchanges
 * s1, s2 are the configurations at beta_i and beta_{i+1} when pair i came up.
 * Uses: the acceptance estimate mean(min(1, e^lnA)) over updates (lower
 * variance than counting accepted swaps) and tuning of the cooling parameter.
 * All zero before the first update; not saved by pt_save. */
pt_status pt_get_exchange_log(pt_handle h, double *lnA, double *lnJ);

/* Copy the configuration at (sample, copy, replica b) to / from the host as
 * double [L^3][3] in natural site order.  pt_set_spins scales every spin
 * whose squared length differs from 1 by more than 1e-6 to unit length (the
 * updates' renormalisation only corrects rounding errors; PT_ERR_ARG for a
 * zero or non-finite spin) and marks the energies for recomputation. */
pt_status pt_get_spins(pt_handle h, int sample, int copy, int replica, double *xyz);
pt_status pt_set_spins(pt_handle h, int sample, int copy, int replica, const double *xyz);

/* Replace the inverse temperatures (host double, same layout as at creation)
 * and/or the cooling parameters (host float [n_samples][n_replicas-1]); either
 * may be NULL.  The values are validated, staged in pinned memory owned by the
 * engine and copied on the engine's stream (ordered before later work); the
 * call does not synchronise and the caller's arrays may be reused at once. */
pt_status pt_set_params(pt_handle h, const double *betas, const float *eps);

/* Set / read the Philox step counter. */
pt_status pt_set_rng_step(pt_handle h, uint64_t step);
pt_status pt_get_rng_step(pt_handle h, uint64_t *step);

/* Save / restore the whole chain state (spins, maps, counters, energies,
 * parameters, step counter) to / from a file.  pt_load needs a handle created
 * with the same shapes and precision.  Resuming is exact: k cycles, save,
 * load, k cycles give the same state as 2k cycles. */
pt_status pt_save(pt_handle h, const char *path);
pt_status pt_load(pt_handle h, const char *path);

/* Per-kernel-class timing on the engine's stream.
 * pt_profile(h, 1) starts recording a CUDA event before and after every
 * kernel launch of the handle (and clears earlier records); pt_profile(h, 0)
 * stops.  pt_profile_read synchronises and returns, per class, the summed
 * event time in milliseconds and the number of kernel launches since the
 * last pt_profile call (launches are counted even while recording is off).
 * Arrays have PT_KERNEL_KINDS entries; either may be NULL. */
typedef enum {
    PT_KERNEL_HB = 0,        /* heat-bath half sweeps */
    PT_KERNEL_OR = 1,        /* overrelaxation half sweeps */
    PT_KERNEL_ENERGY = 2,    /* energy reduction and finalisation */
    PT_KERNEL_EXCHANGE = 3,  /* tempering updates */
    PT_KERNEL_MEASURE = 4,   /* overlap reduction */
    PT_KERNEL_OTHER = 5,     /* initial spins, step counter */
    PT_KERNEL_RESIDENT = 6,  /* whole sweep blocks of a replica held in shared memory */
    PT_KERNEL_KINDS = 7
} pt_kernel_kind;
pt_status pt_profile(pt_handle h, int enable);
pt_status pt_profile_read(pt_handle h, double *ms, int64_t *launches);

/* Choose how pt_sweep runs the local updates.
 *   PT_POLICY_AUTO (default): shared-memory resident sweep blocks when every
 *     sample's replica fits one CTA or a cluster of 2, 4 or 8 CTAs (float: L/2
 *     a multiple of 2 or 4; double: L/2 even; spins and couplings of a replica,
 *     or of its z-slab, at most 200 KB per CTA: float up to L = 16 on one CTA,
 *     L = 24 and 32 on clusters), else streaming half sweeps;
 *   PT_POLICY_STREAMING: one kernel per half sweep over HBM;
 *   PT_POLICY_RESIDENT: resident blocks; PT_ERR_STATE if a sample does not fit.
 * Both give the same chain (same updates, same random numbers). */
typedef enum { PT_POLICY_AUTO = 0, PT_POLICY_STREAMING = 1, PT_POLICY_RESIDENT = 2 } pt_policy;
pt_status pt_set_policy(pt_handle h, int policy);

/* Bounded device-side waits and a hook to test their failure path.
 * The kernels that wait on the device are those that move data with TMA bulk
 * copies and wait for them on an mbarrier: the resident sweep blocks (one CTA
 * or a cluster per replica; their replica's load), the staged heated-proposal
 * pass of the cooling/heating exchange, and the bulk-copy (TMA) half sweep of
 * overrelaxation (selected by PT_TMA=1 in the environment when the handle is
 * created; FP32, every L a multiple of 8, streaming policy).  Each wait polls
 * at most `limit` times (0 restores the default, 2^22), then sets the handle's
 * device error word, gives the copies in flight a bounded chance to land and
 * skips the work that needed them: a resident block leaves its replica in
 * global memory as it was (a cluster does so as a whole), the half sweep
 * leaves the replicas it did not reach; every spin stays a valid unit vector.
 * The next call that synchronises (pt_measure, pt_get_spins, pt_get_stats,
 * ...) returns PT_ERR_TIMEOUT once and clears the word; the handle stays
 * usable.  inject != 0 makes CTA 0 of every later launch of those kernels
 * leave its copies un-issued (for the half sweep: one stage of the first
 * replica of its first work item), so its wait runs out; inject = 0 turns that
 * off.  PT_ERR_STATE if inject != 0 and the handle currently runs none of
 * them (no resident sample and no bulk-copy half sweep). */
pt_status pt_set_wait_limit(pt_handle h, unsigned long long limit, int inject);

/* Energies H = -sum_<xy> J_xy s_x . s_y of configurations that live in the
 * caller's own device memory, computed without allocating any memory.
 * For callers that cannot let a library call cudaMalloc: code embedded in
 * another framework whose memory pool must account for every device byte,
 * and latency-critical loops that forbid allocation after start-up (cudaMalloc
 * may synchronise the device and has no bounded latency).  The paper has no
 * counterpart; this is a service of the library, not a step of the method.
 *   d_spins      device, n_configs configurations, each [L^3][3] in natural
 *                site order, float (PT_FP32) or double (PT_FP64)
 *   precision    PT_FP32 or PT_FP64, the element type of d_spins
 *   L            lattice size, 2 <= L <= 512 (natural order: odd L allowed)
 *   n_configs    number of configurations, >= 0
 *   d_couplings  device float [3][L^3], J[mu][x] of bond (x, x + e_mu),
 *                shared by all configurations
 *   d_energy     device double [n_configs], written (sums in double)
 *   stream       cudaStream_t to enqueue on (NULL: legacy stream); the call
 *                does not synchronise
 * Scratch: the partial sums live in one fixed array of 65536 doubles
 * (512 KiB) in the library's device image, which every GPU that loads the
 * library holds until the process exits.  A call needs
 * n_configs * ceil(L^3 / 2048) entries (at most 32768 configurations at
 * L = 16, 4096 at L = 32); larger requests return PT_ERR_ARG and do nothing.
 * Every call writes each entry it reads, so no clearing is needed, but all
 * calls share the array: calls that overlap on the GPU (other streams or
 * other host threads on the same device) race, and the caller must order
 * them.  The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Errors: PT_ERR_ARG for bad arguments,
 * PT_ERR_CUDA for a failed launch (text in pt_last_error). */
pt_status pt_energy_noalloc(const void *d_spins, int precision, int L, int n_configs,
                            const float *d_couplings, double *d_energy, void *stream);

/* Measured throughput of the shared-memory data path of the current device,
 * the unit that bounds the resident sweep blocks (a resident replica runs
 * every half sweep out of shared memory); it is the peak their roofline is
 * taken against.  Not a step of the method: a probe of the hardware.
 * Every SM runs two 512-thread CTAs streaming conflict-free 16-byte loads over
 * 32 KB of shared memory (about 1 ms); the best of three timed launches on
 * `stream` (cudaStream_t, NULL: legacy stream) is returned, each output may be
 * NULL: bytes_per_s (all SMs), bytes_per_clock_sm (per SM and SM clock) and
 * sm_mhz (the SM clock the probe ran at, from clock64 and the global timer).
 * Synchronises the stream.  Allocates about 160 KB of device memory for the
 * duration of the call.  Errors: PT_ERR_NOMEM, PT_ERR_CUDA. */
pt_status pt_smem_bandwidth(void *stream, double *bytes_per_s, double *bytes_per_clock_sm, double *sm_mhz);

/* Enqueue n_cycles update cycles: a block of local updates (n_hb heat-bath
 * sweeps and n_or overrelaxation sweeps, or n_or_samples[s] for sample s when
 * n_or_samples is not NULL), one tempering update with the stored cooling
 * parameters, and with measure != 0 the overlap reduction into the engine's
 * buffers (read them with pt_measure).  When the engine runs on its own
 * stream and profiling is off, one cycle is captured into a CUDA graph (again
 * whenever the arguments or the kernel paths change) and replayed n_cycles
 * times; the chain is the same as with the individual calls. */
pt_status pt_cycles(pt_handle h, int n_cycles, int n_hb, int n_or, const int *n_or_samples,
                    pt_mode mode, int measure);

/* Autotuner: for every lattice size of the batch, time each candidate way of
 * running the sweeps (shared-memory resident blocks -- one CTA, a cluster of
 * 1024-thread CTAs, or a "narrow" cluster of 512-thread CTAs, two per SM --
 * or streaming half sweeps, with 4, 2 or 1 sites per thread where the row
 * length allows) on the batch itself, a warm-up and two blocks of
 * n_hb + n_or sweeps each, and keep the fastest under PT_POLICY_AUTO.  The
 * chain state (spins, energies, step counter) is restored, so tuning does not
 * change the chain.  Optional host outputs per sample: choice[s] in the
 * encoding of pt_get_paths, best_ms[s] = time of one block with the chosen
 * path.  Allocates a temporary copy of the spins on the device. */
pt_status pt_autotune(pt_handle h, int n_hb, int n_or, int *choice, double *best_ms);

/* The sweep path of every sample now (host int [n_samples]): the vector
 * width (sites per thread: 4, 2 or 1) for streaming half sweeps, + 10 for the
 * resident kernels with one CTA or a cluster of 1024-thread CTAs, + 20 for a
 * narrow cluster of 512-thread CTAs; ctas[s] (host int [n_samples] or NULL)
 * = CTAs per replica (0 when streaming).  PT_CL_NARROW=1 in the environment
 * when the handle is created selects narrow clusters wherever they exist,
 * until pt_autotune decides. */
pt_status pt_get_paths(pt_handle h, int *choice, int *ctas);

/* Set the sweep path of every sample from codes in the encoding of
 * pt_get_paths (host int [n_samples]), e.g. the choices of an earlier
 * pt_autotune of the same batch shape kept in a cache, under
 * PT_POLICY_AUTO.  Nothing changes if a code is not a path of its sample:
 * PT_ERR_ARG for a malformed code or a vector width the row length does not
 * allow, PT_ERR_STATE for a resident shape the sample does not fit.  The
 * chain is unchanged (every path runs the same updates). */
pt_status pt_set_paths(pt_handle h, const int *choice);

/* Release all device memory of the handle.  NULL is accepted. */
pt_status pt_destroy(pt_handle h);

/* ---------------------------------------------------------------------------
 * Learned ladder.  A perceptron 4 -> 64 -> 64 -> 2P+1 (ReLU hidden layers,
 * bfloat16 weights, float accumulation, float master weights) maps the
 * description of a sample to the parameters of its tempering: the shape of
 * the inverse-temperature ladder, the cooling/heating parameter epsilon of
 * every pair and the number of replicas the range needs.  Section III.B
 * motivates it (the best epsilon depends on the pair of temperatures and
 * decreases with beta_{i+1}/beta_i; one epsilon for all pairs was the paper's
 * simplification), and section IV.A suggests tuning epsilon per pair.  The net only chooses parameters: the chain is exact for every
 * ladder.  The paper has no network; the design is this library's.
 *
 * Features x (float [4] per row): ln L, beta_min, beta_max, and the coupling
 * statistic g = mean_x sqrt(sum_y J_xy^2) / (sqrt(6) rms J).
 * Outputs z (float [2P+1] per row), with P knots u_k = k / P:
 *   d_k = softplus(z_k) + PT_MLP_SHAPE_FLOOR, f_k = d_k / sum_j d_j,
 *   F(u_k) = sum_{j<k} f_j, F linear between knots (F(u) = u is the
 *   geometric ladder; the floor keeps every ladder strictly ascending);
 *   ln beta_i = ln beta_min + F(i / (NT - 1)) ln(beta_max / beta_min);
 *   e_k = sigmoid(z_{P+k}), kappa(u) = kappa_max e(u), e linear between the
 *   knot midpoints (k + 1/2) / P, constant beyond the outer ones;
 *   eps_i = kappa((i + 1/2) / (NT - 1)) (ln beta_{i+1} - ln beta_i);
 *   Lambda = exp(z_{2P}), the predicted sum over the pairs of an
 *   equal-acceptance ladder of the width sigma of the Gaussian log acceptance
 *   ratio (acceptance erfc(sigma / 2^{3/2})); NT = 1 + ceil(Lambda /
 *   sigma_target) replicas give each pair the acceptance of sigma_target.
 * Targets t (float [2P+1] per row): t_k = target f_k (summing to 1),
 * t_{P+k} = target e_k in (0, 1), t_{2P} = target ln Lambda.  Loss of a row:
 *   (1/P) sum_k [ (P (f_k - t_k))^2 + w_kappa (e_k - t_{P+k})^2 ]
 *   + (z_{2P} - t_{2P})^2,
 * averaged over the batch.  Parameters (float, pt_mlp_num_params of them):
 * [W1 64x4 | b1 64 | W2 64x64 | b2 64 | W3 (2P+1)x64 | b3 2P+1], W[out][in].
 * All arrays of these calls are HOST arrays; the calls copy them to and from
 * the device and synchronise the handle's stream before returning.
 * ------------------------------------------------------------------------- */
#define PT_MLP_IN 4
#define PT_MLP_HIDDEN 64
#define PT_MLP_MAX_KNOTS 64
#define PT_MLP_SHAPE_FLOOR 0.01f
typedef struct pt_mlp *pt_mlp_handle;

/* Create a net with n_knots (1..PT_MLP_MAX_KNOTS) knots on the given
 * cudaStream_t (NULL: legacy stream).  Weights are initialised from seed
 * (splitmix64, uniform in +-1/sqrt(fan_in), the last layer scaled by 0.01 so
 * that a fresh net proposes a nearly geometric ladder); biases are zero.
 * Errors: PT_ERR_ARG, PT_ERR_NOMEM, PT_ERR_CUDA. */
pt_status pt_mlp_create(pt_mlp_handle *out, int n_knots, uint64_t seed, void *stream);

/* Number of float parameters (0 for NULL). */
int pt_mlp_num_params(pt_mlp_handle h);

/* Replace the master weights (host float [num_params]) and refresh the
 * bfloat16 copy; the Adam moments and step count are reset.  PT_ERR_ARG for
 * a non-finite value. */
pt_status pt_mlp_set_params(pt_mlp_handle h, const float *params);

/* Read the master weights (float) and/or the bfloat16 copy used by the
 * products (raw bits); either pointer may be NULL. */
pt_status pt_mlp_get_params(pt_mlp_handle h, float *params, uint16_t *bf16);

/* Forward pass of batch rows: x float [batch][4] -> z float [batch][2P+1]. */
pt_status pt_mlp_forward(pt_mlp_handle h, int batch, const float *x, float *z);

/* Loss and its gradient with respect to the master weights (float
 * [num_params], computed through the bfloat16 weights).  loss or grad may be
 * NULL.  w_kappa >= 0 weights the epsilon part of the loss. */
pt_status pt_mlp_loss_grad(pt_mlp_handle h, int batch, const float *x, const float *target, float w_kappa,
                           float *loss, float *grad);

/* steps full-batch Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, learning
 * rate lr) on the device.  losses (float [steps], may be NULL) receives the
 * loss before each step; asking for it synchronises every step. */
pt_status pt_mlp_train(pt_mlp_handle h, int batch, const float *x, const float *target, float w_kappa, int steps,
                       float lr, float *losses);

/* Ladders proposed for batch rows.  Row r has n_temps[r] inverse
 * temperatures between beta_min[r] and beta_max[r] (0 < beta_min < beta_max),
 * written to betas[r * stride + i] (double, strictly ascending, exactly
 * beta_min and beta_max at the ends), and n_temps[r] - 1 values epsilon to
 * eps[r * (stride - 1) + i] (float); unused entries are zero.  n_temps is in
 * and out: 2 <= n_temps[r] <= stride is used as given; n_temps[r] <= 0 asks
 * the net, NT = 1 + ceil(Lambda / sigma_target) clamped to [2, stride], and
 * the count chosen is written back (sigma_target > 0 is then required).
 * kappa_max >= 0 scales the epsilon outputs.  stride >= 2. */
pt_status pt_mlp_ladder(pt_mlp_handle h, int batch, const float *x, const double *beta_min, const double *beta_max,
                        int *n_temps, int stride, float kappa_max, double sigma_target, double *betas,
                        float *eps);

/* Release the net.  NULL is accepted. */
pt_status pt_mlp_destroy(pt_mlp_handle h);

/* Text of the calling thread's last error ("" if none). */
const char *pt_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PT_H */
