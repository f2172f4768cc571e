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


def _lattice_graph(L):
    """The periodic L^3 lattice as a graph: {(x, y): [(mu, x'), ...]} with
    x < y, listing the bonds (mu, x') that join the two sites (two of them
    for every neighbour pair at L = 2, where they act as one bond of coupling
    J_eff = their sum; one otherwise)."""
    N = L ** 3

    def step(x, mu):
        c = [x % L, (x // L) % L, x // (L * L)]
        c[mu] = (c[mu] + 1) % L
        return c[0] + L * (c[1] + L * c[2])

    g = {}
    for x in range(N):
        for mu in range(3):
            y = step(x, mu)
            g.setdefault((min(x, y), max(x, y)), []).append((mu, x))
    return g


def _simple_cycles(L, max_len=6):
    """Every simple cycle (closed walk through distinct sites) of at most
    max_len edges of the lattice graph, once each, as a list of edge keys."""
    g = _lattice_graph(L)
    adj = {}
    for (x, y) in g:
        adj.setdefault(x, []).append(y)
        adj.setdefault(y, []).append(x)
    out = []
    for v in sorted(adj):
        stack = [(v, [v])]
        while stack:
            x, path = stack.pop()
            for y in adj[x]:
                if y == v and len(path) >= 3 and path[1] < path[-1]:
                    cyc = path + [v]
                    out.append([(min(a, b), max(a, b)) for a, b in zip(cyc[:-1], cyc[1:])])
                elif y > v and y not in path and len(path) < max_len:
                    stack.append((y, path + [y]))
    return out


def _series_parts(L, J, beta):
    """ln Z of the high-temperature expansion, through the graphs of six
    bonds (each bond weight e^{u s.s'} expanded in Legendre polynomials,
    u = beta J, with the single-bond factors ln(sinh u / u) kept exactly):
    every simple cycle C contributes 3 prod_{b in C} t(u_b), t = Langevin
    function (the vertex integrals of the l = 1 terms around the loop).  On
    the L = 3 lattice the winding cycles have three bonds, which brings two
    more terms of order u^6 on each of them: the loop of l = 2 terms,
    5 prod a2(u_b) with a2 = 1 - 3 t(u)/u, and the cumulant -(3 prod t)^2 / 2
    (a loop cannot be occupied twice).  Loops that share only a site
    contribute the product of their weights to Z, so they cancel in ln Z.
    Returns (single-bond part, cycles of fewer than six bonds, the six-bond
    order) as functions of beta."""
    g = _lattice_graph(L)
    Je = {k: sum(J[mu, x] for mu, x in bonds) for k, bonds in g.items()}
    cycles = _simple_cycles(L, 6)

    def t_of(b, k):
        return langevin(np.array([b * Je[k]]))[0]

    def a2_of(b, k):
        u = b * Je[k]
        return u * u / 15.0 if abs(u) < 1e-3 else 1.0 - 3.0 * langevin(np.array([u]))[0] / u

    def low(b):
        return sum(3 * np.prod([t_of(b, k) for k in c]) for c in cycles if len(c) < 6)

    def six(b):
        v = sum(3 * np.prod([t_of(b, k) for k in c]) for c in cycles if len(c) == 6)
        if L == 3:
            for c in (c for c in cycles if len(c) == 3):
                w = 3 * np.prod([t_of(b, k) for k in c])
                v += 5 * np.prod([a2_of(b, k) for k in c]) - 0.5 * w * w
        return v

    Jv = np.array(list(Je.values()))
    return (lambda b: -(Jv * langevin(b * Jv)).sum()), low, six


def _ddb(f, b, h=1e-5):
    return (f(b + h) - f(b - h)) / (2 * h)


def _highT_energy(L, J, beta):
    """<H> = -d ln Z / d beta of the series through six-bond graphs."""
    single, low, six = _series_parts(L, J, beta)
    return single(beta) - _ddb(low, beta) - _ddb(six, beta)


def _highT_remainder(L, J, beta):
    """Allowance for the graphs left out: the size of the six-bond order's
    contribution to <H>.  The first omitted orders are eight-bond graphs
    (L = 2, 4; smaller than the six-bond order by about (beta J / 3)^2 times
    the ratio of their counts, 0.1 at beta = 0.3) and seven-bond cycles
    (L = 3; about beta |J| / 3 times the lattice's growth constant of cycles,
    below 0.5 at beta = 0.3), so the six-bond order bounds them with margin."""
    _, _, six = _series_parts(L, J, beta)
    return abs(_ddb(six, beta))


@pytest.mark.parametrize("L,order", [(2, 0), (4, 0), (3, 1)])
def test_high_temperature_series(orc, L, order):
    J = W.couplings(L, 70 + L).astype(np.float64)
    betas = np.array([0.1, 0.2, 0.3])
    run = orc.Run(L, J, betas, n_copies=2, seed=5 + L)
    n = 24000 if L <= 3 else 16000
    Hs, _, _ = run.cycles(n, n_hb=1, n_or=1, mode=0, order=order)
    m, e = block_mean_err(Hs[n // 10:].reshape(-1, 2 * 3).reshape(-1, 2, 3).mean(1))
    for b, beta in enumerate(betas):
        ref = _highT_energy(L, J, beta)
        assert abs(m[b] - ref) < 4.5 * e[b] + _highT_remainder(L, J, beta), (L, beta, m[b], ref, e[b])


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


def test_exactness_check_detects_wrong_jacobians(orc):
    """Power of the exactness check above (same lattice, couplings, ladder,
    cooling parameter and run length).  The cooling/heating acceptance is run
    with the Jacobian of the heated configuration taken where section III.B's
    printed formula, read literally, puts it (at s2 itself instead of at its
    pre-image C^-1 s2), and with no Jacobian at all.  Both break detailed
    balance; the check must see each of them: <H>(beta) at some temperature
    more than 6 combined standard errors from the standard swap's (the check
    passes the correct placement at 4.5)."""
    L = 2
    J = W.couplings(L, 90).astype(np.float64)
    betas = np.array([0.8, 1.3, 1.9, 2.6])
    n = 30000

    def mean_H(mode, variant):
        with orc.jacobian_variant(variant):
            run = orc.Run(L, J, betas, n_copies=2, seed=100 + mode, eps=0.06)
            Hs, _, _ = run.cycles(n, n_hb=1, n_or=1, mode=mode)
        return block_mean_err(Hs[n // 10:].mean(1))

    m0, e0 = mean_H(0, 0)
    for variant in (1, 2):
        m, e = mean_H(2, variant)
        z = np.abs(m - m0) / np.sqrt(e ** 2 + e0 ** 2)
        assert z.max() > 6.0, (variant, z)
    # the hook is reset on leaving the context: the correct placement again
    m, e = mean_H(2, 0)
    assert within(m, e, m0, e0, 4.5).all()
