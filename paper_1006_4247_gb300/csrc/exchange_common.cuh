// exchange_common.cuh -- helpers shared by the exchange kernels.
#pragma once
#include "kernels.h"
#include "pt_device.cuh"

namespace ptk {

// Metropolis acceptance (section I, Eq. 1) from ln A and ln u.
__device__ __forceinline__ bool accept_lnu(double lnA, double lnu) { return lnA >= 0.0 || lnu < lnA; }

// Record a pair's log acceptance ratio and, for cooling/heating, its two
// Jacobian terms (read back by pt_get_exchange_log).
__device__ __forceinline__ void xlog_write(const DevBatch& a, long long pair, double lnA, double lj1, double lj2) {
    double* p = a.xlog + 3 * pair;
    p[0] = lnA;
    p[1] = lj1;
    p[2] = lj2;
}

// Per-pair constants of the decimation ratio (section III.A, Appendix A),
// computed once per launch in double and rounded to the sweep precision T:
// beta_b, beta_{b+1} - beta_b and ln(beta_{b+1} / beta_b) (0 when
// beta_b = 0).  The caller synchronises the block before reading them.
template <typename T, int N>
struct DecimPairs {
    T b[N], db[N], lr[N];
    __device__ void load(const double* beta, int NT) {
        for (int q = (int)threadIdx.x; q < NT; q += (int)blockDim.x) {
            const double b1 = beta[q];
            b[q] = (T)b1;
            if (q + 1 < NT) {
                const double b2 = beta[q + 1];
                db[q] = (T)(b2 - b1);
                lr[q] = b1 > 0.0 ? (T)log(b2 / b1) : (T)0;
            }
        }
    }
};

// The parts of a chain's tempering update that do not depend on the walk's
// decisions, prepared by the whole block before the walk so that the one
// thread that decides each pair waits on neither memory, Philox nor a double
// exponential: ln u of every pair's uniform (purpose 1, c0 = pair, c1 = copy;
// the same numbers the decision would draw) and a per-pair count of
// acceptances, added to the global counters once after the walk.  The test
// u < e^{ln A} is taken as ln u < ln A (the same decision up to the rounding
// of one logarithm).
template <int N>
struct PairDraws {
    double lnu[N];
    int acc[N];
    __device__ void load(uint64_t seed, uint32_t sample, uint32_t copy, unsigned long long step, int n_pairs) {
        for (int i = (int)threadIdx.x; i < n_pairs; i += (int)blockDim.x) {
            const uint4 w = rng_words(seed, sample, (uint32_t)i, copy, step, 1u);
            lnu[i] = log(u53(w.x, w.y));  // u = 0 gives -inf: always below ln A
            acc[i] = 0;
        }
    }
    // every pair was proposed once; the caller synchronises the block first
    __device__ void store(long long* prop, long long* accg, int n_pairs) const {
        for (int i = (int)threadIdx.x; i < n_pairs; i += (int)blockDim.x) {
            prop[i] += 1;
            accg[i] += acc[i];
        }
    }
};

}  // namespace ptk
