"""Shared helpers of the GPU tests: engine construction from seeded inputs and
element-wise comparison with the oracle."""
import numpy as np

import oracle as orc
from paper_1006_4247_gb300 import pt
from paper_1006_4247_gb300 import workloads as W


def site_colour(L):
    x = np.arange(L ** 3)
    return ((x % L) + (x // L) % L + x // (L * L)) % 2


def make_engine(L, S=1, NT=4, C=2, precision="fp64", seed=11, jseed=100, bmin=0.5, bmax=2.0,
                start="random"):
    J = np.stack([W.couplings(L, jseed + s) for s in range(S)])
    B = np.stack([W.linear_betas(NT, bmin, bmax) for _ in range(S)])
    eng = pt.Engine(L, J, B, n_copies=C, precision=precision, seed=seed, start=start)
    return eng, J.astype(np.float64), B


def set_random_state(eng, S, C, NT, L, seed):
    """Put seeded random unit spins into every replica; return them as the
    engine stores them (rounded to the engine's precision)."""
    st = np.zeros((S, C, NT, L ** 3, 3))
    for s in range(S):
        for c in range(C):
            for b in range(NT):
                v = W.random_spins(L, seed + 1000 * s + 100 * c + b)
                eng.set_spins(s, c, b, v)
                st[s, c, b] = eng.get_spins(s, c, b)
    return st


def get_state(eng, S, C, NT):
    return np.stack([np.stack([np.stack([eng.get_spins(s, c, b) for b in range(NT)])
                               for c in range(C)]) for s in range(S)])


def ambiguous_basis_sites(L, J, s, colour, tol=1e-4):
    """Sites of `colour` whose neighbour field is nearly perpendicular to e_z:
    there the heat-bath basis of float and double arithmetic may pick
    opposite orientations (sign of S_z), so only the component along S and
    |s| = 1 are unique."""
    out = np.zeros(L ** 3, bool)
    col = site_colour(L)
    for x in np.nonzero(col == colour)[0]:
        S = orc.local_field(L, J, s, x)
        n = np.linalg.norm(S)
        out[x] = n == 0 or abs(S[2]) < tol * n
    return out
