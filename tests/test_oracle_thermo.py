"""Statistical pins of the oracle's whole update cycle: closed forms at
beta = 0, the high-temperature series of <H>, and exactness of the two
modified exchanges of section III (they must sample the same ensemble as the
standard swap)."""
import numpy as np
import pytest

from paper_1006_4247_gb300 import workloads as W
from statutil import block_mean_err, within


def langevin(u):
    u = np.asarray(u, float)
    out = np.empty_like(u)
    small = np.abs(u) < 1e-4
    out[small] = u[small] / 3 - u[small] ** 3 / 45
    us = u[~small]
    out[~small] = 1 / np.tanh(us) - 1 / us
    return out


def test_beta_zero_closed_forms(orc):
    """At beta = 0 every heat-bath sweep draws fresh uniform spins:
    <H> = 0, Var H = sum_b J_b^2 / 3, <chi> = 1."""
    L = 4
    J = W.couplings(L, 61).astype(np.float64)
    run = orc.Run(L, J, np.array([0.0, 0.0]), n_copies=2, seed=17)
    n = 3000
    Hs, chis, _ = run.cycles(n, n_hb=1, n_or=0, mode=0)
    H = Hs.reshape(-1)
    var_exact = (J ** 2).sum() / 3
    assert abs(H.mean()) < 5 * np.sqrt(var_exact / H.size)
    assert abs(H.var() - var_exact) < 5 * np.sqrt(2.0 / H.size) * var_exact
    chi = chis.reshape(-1)
    assert abs(chi.mean() - 1.0) < 5 * chi.std() / np.sqrt(chi.size)


def _cycles_L(L):
    """Closed loops of bonds at the lowest orders: plaquettes, and for L <= 4
    the loops that wind around the periodic lattice.  Each loop is a list of
    (mu, x) bonds."""
    N = L ** 3

    def idx(i, j, k):
        return (i % L) + L * ((j % L) + L * (k % L))

    def step(x, mu):
        i, j, k = x % L, (x // L) % L, x // (L * L)
        d = [0, 0, 0]
        d[mu] = 1
        return idx(i + d[0], j + d[1], k + d[2])

    loops = []
    for x in range(N):
        for mu in range(3):
            for nu in range(mu + 1, 3):
                xm = step(x, mu)
                xn = step(x, nu)
                loops.append([(mu, x), (nu, xm), (mu, xn), (nu, x)])
    if L in (3, 4):
        for mu in range(3):
            for x in range(N):
                i, j, k = x % L, (x // L) % L, x // (L * L)
                if (i, j, k)[mu] != 0:
                    continue
                line, y = [], x
                for _ in range(L):
                    line.append((mu, y))
                    y = step(y, mu)
                loops.append(line)
    return loops


def _highT_energy(L, J, beta):
    """<H> from ln Z = sum_b ln(sinh u_b/u_b) + 3 sum_loops prod_b t(u_b),
    t = Langevin function, u = beta J (expansion in Legendre polynomials of
    each bond weight; the lowest neglected graphs enter <H> at O(beta^5))."""
    loops = _cycles_L(L)

    def loop_part(b):
        t = langevin(b * J)
        return 3 * sum(np.prod([t[mu, x] for mu, x in lp]) for lp in loops)

    h = 1e-5
    d = (loop_part(beta + h) - loop_part(beta - h)) / (2 * h)
    return -(J * langevin(beta * J)).sum() - d


def _highT_energy_L2(J, beta):
    """L = 2: the two bonds of each neighbour pair merge into J_eff; the graph
    is the 3-cube (12 edges, 6 faces)."""
    L = 2

    def idx(i, j, k):
        return (i % 2) + 2 * ((j % 2) + 2 * (k % 2))

    edges = {}
    for x in range(8):
        i, j, k = x % 2, (x // 2) % 2, x // 4
        for mu in range(3):
            d = [0, 0, 0]
            d[mu] = 1
            y = idx(i + d[0], j + d[1], k + d[2])
            key = (min(x, y), max(x, y))
            edges[key] = edges.get(key, 0.0) + J[mu, x]
    faces = []
    for mu in range(3):
        for nu in range(mu + 1, 3):
            for base in range(8):
                bi = [base % 2, (base // 2) % 2, base // 4]
                if bi[mu] or bi[nu]:
                    continue
                corners = []
                for a, b in ((0, 0), (1, 0), (1, 1), (0, 1)):
                    c = list(bi)
                    c[mu] += a
                    c[nu] += b
                    corners.append(idx(*c))
                faces.append([(min(corners[n], corners[(n + 1) % 4]),
                               max(corners[n], corners[(n + 1) % 4])) for n in range(4)])
    assert len(edges) == 12 and len(faces) == 6
    Je = np.array(list(edges.values()))

    def loop_part(b):
        return 3 * sum(np.prod([langevin(np.array([b * edges[e]]))[0] for e in f]) for f in faces)

    h = 1e-5
    d = (loop_part(beta + h) - loop_part(beta - h)) / (2 * h)
    return -(Je * langevin(beta * Je)).sum() - d


@pytest.mark.parametrize("L,order", [(2, 0), (4, 0), (3, 1)])
def test_high_temperature_series(orc, L, order):
    J = W.couplings(L, 70 + L).astype(np.float64)
    betas = np.array([0.1, 0.2, 0.3])
    run = orc.Run(L, J, betas, n_copies=2, seed=5 + L)
    n = 24000 if L <= 3 else 16000
    Hs, _, _ = run.cycles(n, n_hb=1, n_or=1, mode=0, order=order)
    m, e = block_mean_err(Hs[n // 10:].reshape(-1, 2 * 3).reshape(-1, 2, 3).mean(1))
    for b, beta in enumerate(betas):
        ref = _highT_energy_L2(J, beta) if L == 2 else _highT_energy(L, J, beta)
        assert abs(m[b] - ref) < 4.5 * e[b] + 1e-3, (L, beta, m[b], ref, e[b])


def test_modified_exchanges_sample_the_same_ensemble(orc):
    """Standard, decimation and cooling/heating tempering give the same
    <H>(beta) and <chi>(beta) within errors (exactness of the moves)."""
    L = 2
    J = W.couplings(L, 90).astype(np.float64)
    betas = np.array([0.8, 1.3, 1.9, 2.6])
    n = 30000
    res = {}
    for mode in (0, 1, 2):
        run = orc.Run(L, J, betas, n_copies=2, seed=100 + mode, eps=0.06)
        Hs, chis, _ = run.cycles(n, n_hb=1, n_or=1, mode=mode)
        mH, eH = block_mean_err(Hs[n // 10:].mean(1))
        mC, eC = block_mean_err(chis[n // 10:])
        res[mode] = (mH, eH, mC, eC)
    for mode in (1, 2):
        assert within(res[mode][0], res[mode][1], res[0][0], res[0][1], 4.5).all(), mode
        assert within(res[mode][2], res[mode][3], res[0][2], res[0][3], 4.5).all(), mode


def test_modified_exchanges_raise_acceptance(orc):
    """Section IV.A: at equal ladders the decimation and (tuned) cooling/heating
    swaps are accepted more often than the standard swap (trend only)."""
    L = 6
    J = W.couplings(L, 90).astype(np.float64)
    betas = np.linspace(2.0, 3.0, 4)
    acc = {}
    for mode, eps in ((0, 0.0), (1, 0.0), (2, 0.02)):
        run = orc.Run(L, J, betas, n_copies=2, seed=100 + mode, eps=eps)
        run.cycles(200, n_hb=1, n_or=L, mode=mode, record=False)
        run.acc[:] = 0
        run.prop[:] = 0
        run.cycles(1000, n_hb=1, n_or=L, mode=mode, record=False)
        acc[mode] = run.acc.sum(0) / run.prop.sum(0)
    assert (acc[1] > acc[0]).all() and acc[1].mean() > 1.5 * acc[0].mean()
    assert acc[2].mean() > 1.2 * acc[0].mean()
