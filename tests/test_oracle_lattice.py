"""Pins of the oracle's lattice observables: the Hamiltonian of section I, the
neighbour field of Eq. bigS and the overlap of section II, each against an
independent numpy formulation (np.roll on the [k, j, i] grid)."""
import numpy as np
import pytest

from paper_1006_4247_gb300 import workloads as W


def _grid(L, s):
    return s.reshape(L, L, L, 3)  # [k, j, i, a]


def _roll_energy(L, J, s):
    g = _grid(L, s)
    Jg = J.reshape(3, L, L, L)
    H = 0.0
    for mu, axis in enumerate((2, 1, 0)):  # mu = 0 -> i (last grid axis)
        nb = np.roll(g, -1, axis=axis)
        H -= (Jg[mu] * (g * nb).sum(-1)).sum()
    return H


def _roll_field(L, J, s):
    g = _grid(L, s)
    Jg = J.reshape(3, L, L, L)
    S = np.zeros_like(g)
    for mu, axis in enumerate((2, 1, 0)):
        S += Jg[mu][..., None] * np.roll(g, -1, axis=axis)
        S += np.roll(Jg[mu], 1, axis=axis)[..., None] * np.roll(g, 1, axis=axis)
    return S.reshape(-1, 3)


@pytest.mark.parametrize("L", [2, 3, 4, 5])
def test_energy_and_field_vs_roll(orc, L):
    J = W.couplings(L, 10 + L).astype(np.float64)
    s = W.random_spins(L, 20 + L)
    H = orc.energy(L, J, s)
    assert abs(H - _roll_energy(L, J, s)) < 1e-11 * max(1, abs(H))
    S = _roll_field(L, J, s)
    for x in range(L ** 3):
        assert np.allclose(orc.local_field(L, J, s, x), S[x], atol=1e-13)
    # each bond appears twice in sum_x s_x . S_x
    assert abs(-0.5 * (s * S).sum() - H) < 1e-11 * max(1, abs(H))


def test_energy_special_cases(orc):
    L = 4
    N = L ** 3
    J = np.ones((3, N))
    s = np.tile([0.0, 0.0, 1.0], (N, 1))
    assert orc.energy(L, J, s) == -3 * N
    # staggered (antiferromagnetic) on the bipartite lattice: +3N
    x = np.arange(N)
    col = ((x % L) + (x // L) % L + x // (L * L)) % 2
    s2 = s * (1 - 2 * col)[:, None]
    assert orc.energy(L, J, s2) == 3 * N


def test_energy_rotation_invariance(orc, rng):
    from scipy.spatial.transform import Rotation
    L = 4
    J = W.couplings(L, 3).astype(np.float64)
    s = W.random_spins(L, 4)
    Rm = Rotation.random(random_state=7).as_matrix()
    assert abs(orc.energy(L, J, s @ Rm.T) - orc.energy(L, J, s)) < 1e-11


def test_checkerboard_is_bipartite(orc):
    for L in (2, 4, 6):
        N = L ** 3
        for x in range(N):
            i, j, k = x % L, (x // L) % L, x // (L * L)
            for d in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
                y = (i + d[0]) % L + L * ((j + d[1]) % L + L * ((k + d[2]) % L))
                assert orc._load().orc_color(L, x) != orc._load().orc_color(L, y)


def test_overlap(orc, rng):
    from scipy.spatial.transform import Rotation
    L = 4
    N = L ** 3
    s1 = W.random_spins(L, 1)
    s2 = W.random_spins(L, 2)
    Q, chi = orc.overlap(L, s1, s2)
    assert np.allclose(Q, np.einsum("xa,xb->ab", s1, s2), atol=1e-12)
    assert abs(chi - (Q ** 2).sum() / N) < 1e-12
    # chi is invariant under independent global rotations of the two copies
    R1 = Rotation.random(random_state=1).as_matrix()
    R2 = Rotation.random(random_state=2).as_matrix()
    _, chi_r = orc.overlap(L, s1 @ R1.T, s2 @ R2.T)
    assert abs(chi_r - chi) < 1e-10
    # identical aligned copies: Q = diag(N, 0, 0), chi = N
    a = np.tile([1.0, 0.0, 0.0], (N, 1))
    _, chi_a = orc.overlap(L, a, a)
    assert chi_a == N


def test_init_spins(orc):
    L = 6
    s = orc.init_spins(L, 0, 77, 3, 5)
    assert np.allclose(np.linalg.norm(s, axis=1), 1.0, atol=1e-14)
    o = orc.init_spins(L, 1, 77, 3, 5)
    assert (o == np.array([1.0, 0.0, 0.0])).all()
