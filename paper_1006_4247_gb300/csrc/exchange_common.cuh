// exchange_common.cuh -- helpers shared by the exchange kernels.
#pragma once
#include "pt_device.cuh"

namespace ptk {

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

}  // namespace ptk
