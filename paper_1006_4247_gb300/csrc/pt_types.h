// pt_types.h -- descriptors shared by the host engine and the kernels.
//
// Device layout (all arrays live in one engine allocation set):
//   spins   per chain (sample, copy) a pool of NT + 2 buffers; buffer p of
//           chain ch starts at chain_off[ch] + p * 3N elements (float or
//           double).  A buffer is colour-split structure-of-arrays:
//           [colour c][component a][h], h = ih + (L/2)(j + L k), ih = i >> 1,
//           so site (i,j,k) of colour c sits at h with i = 2 ih + ((j+k+c)&1).
//           NT buffers hold the live configurations; two are scratch for the
//           cooling/heating exchange.
//   J       per sample, colour-split forward couplings [colour][mu][h]:
//           the coupling of bond (x, x + e_mu) for the colour-c site x at h.
//           The backward bond of x is the forward bond of its colour-(1-c)
//           neighbour x - e_mu, read at that neighbour's h.
//   replica r = (chain ch, beta index b) = chain_r0[ch] + b; bufmap[r] is the
//           physical buffer holding the configuration now at beta index b,
//           label[r] its identity (for round trips), H[r] its energy.
#pragma once
#include <stdint.h>

namespace ptk {

// Division by a runtime constant d >= 1 for numerators 0 <= n < 2^31:
// q = umulhi(n, m) >> s with m = ceil(2^(31+l) / d), l = ceil(log2 d),
// s = l - 1 (Granlund & Montgomery, PLDI'94).  d == 1 is flagged by m == 0.
struct FastDiv {
    uint32_t d, m, s, pad;
};

struct SampleDesc {
    int L, hL, half, NT;      // L, L/2, L^3/2, replicas per copy
    FastDiv div_hL, div_L;
    long long J_off;          // float offset of this sample's colour-split J
    int beta_off;             // first beta of this sample in betas[]
    int eps_off;              // first eps (NT - 1 per sample)
    int chain0;               // first chain of this sample
    int r0;                   // first replica of chain0
    int tile0;                // first half-sweep tile of replica r0
    int tiles_per_rep;        // ceil(half / (TILE * vec))
    int vec;                  // sites per thread in the half sweep (4, 2 or 1)
    int tma_planes;           // z planes per item of the bulk-copy half sweep (0: not used)
    int resident;             // CTAs per replica of the shared-memory resident sweeps (0: streaming)
    int narrow;               // 1: clusters of 512-thread CTAs, two per SM (resident > 1 only)
};

struct ChainDesc {
    int s, copy, r0, pair_off;   // sample, copy, first replica, first pair counter
};

constexpr int TILE = 256;        // threads per half-sweep tile (a tile is TILE * vec sites)

}  // namespace ptk
