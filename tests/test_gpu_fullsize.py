"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times, on sampled outputs the oracle computes one by one:

  L = 16, 64 samples x 24 replicas x 2 copies, float (one CTA per replica in
  shared memory, staged cooling/heating exchange);
  L = 32, 16 samples x 48 replicas x 2 copies, float (clusters of CTAs per
  replica, narrow ones of 8 CTAs where the autotuner picks them as it does on
  GB300; cluster decimation exchange);
  the uneven batch of 256 samples, L from {8, 12, 16, 24, 32}, 5L/4
  overrelaxation sweeps per sample (one CTA or narrow clusters by size).

The engines run the autotuner first, as bench.py does, so the paths checked
are the ones it times (the tests assert which).

Checked per sampled replica: one heat-bath sweep and one overrelaxation sweep
site by site (the second half sweep from the engine's first-half result, as
in the small parity tests), energy conservation of a whole block of
overrelaxation sweeps, |s| = 1, the engine energy against the oracle's H, and
one exchange of sampled chains against the oracle's decisions.
"""
import numpy as np
import pytest

import oracle as orc
from gpu_util import ambiguous_basis_sites, check_float_walk, exchange_walk, float_tolerances, site_colour
from paper_1006_4247_gb300 import pt
from paper_1006_4247_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1006_4247_gb300 import _build
    _build.build()


def _engine(name):
    w = W.WORKLOADS[name]()
    J = np.stack(w.couplings())
    B = np.stack(w.betas())
    eng = pt.Engine(w.L[0], J, B, n_copies=2, precision="fp32", seed=7)
    eps = np.concatenate([np.full(n - 1, w.eps, np.float32) for n in w.n_replicas])
    eng.set_params(eps=eps)
    eng.autotune(w.n_hb, w.n_or)
    return w, eng, J.astype(np.float64), B


# resident paths (pt_get_paths codes >= 10) at both sizes; at L = 32 the
# autotuner's pick between wide and narrow clusters is the one checked
EXPECTED_PATH = {"L16_R24_S64": (10,), "L32_R48_S16": (10, 20)}


def _check_half_sweeps(L, J, before, after, kind, beta, seed, sample, rep_id, step0):
    col = site_colour(L)
    cur = before.copy()
    for colour in (0, 1):
        if kind == "hb":
            ref = orc.hb_halfsweep(L, J, cur, colour, beta, seed, sample, rep_id, step0 + colour)
            amb = ambiguous_basis_sites(L, J, cur, colour)
        else:
            ref = orc.or_halfsweep(L, J, cur, colour)
            amb = np.zeros(L ** 3, bool)
        m = (col == colour) & ~amb
        assert np.abs(after[m] - ref[m]).max() <= 1e-5, (kind, colour)
        for x in np.nonzero((col == colour) & amb)[0]:
            Sx = orc.local_field(L, J, cur, x)
            n = Sx / np.linalg.norm(Sx)
            assert abs(after[x] @ n - ref[x] @ n) <= 1e-5
        cur = cur.copy()
        cur[col == colour] = after[col == colour]


@pytest.mark.parametrize("name,samples", [
    ("L16_R24_S64", [(0, 0, 0), (33, 1, 11), (63, 1, 23)]),
    ("L32_R48_S16", [(0, 0, 0), (9, 1, 30), (15, 0, 47)]),
])
def test_fullsize_sweeps_sampled(name, samples):
    w, eng, J, B = _engine(name)
    L = w.L[0]
    NT = w.n_replicas[0]
    choice, _ = eng.paths()
    assert all(c // 10 * 10 in EXPECTED_PATH[name] for c in choice), choice
    eng.sweep(w.n_hb, w.n_or)          # one cycle exactly as the benchmark runs it
    eng.exchange(w.exchange)
    for kind, (nh, no) in (("hb", (1, 0)), ("or", (0, 1))):
        before = {t: eng.get_spins(*t) for t in samples}
        step0 = eng.step
        eng.sweep(nh, no)
        for (s, c, b) in samples:
            after = eng.get_spins(s, c, b)
            _check_half_sweeps(L, J[s], before[(s, c, b)], after, kind, B[s, b], 7, s, c * NT + b, step0)
            assert np.allclose(np.linalg.norm(after, axis=1), 1.0, atol=1e-5)
    # a whole overrelaxation block conserves every replica's energy
    H0 = eng.energies()
    eng.sweep(0, w.n_or)
    H1 = eng.energies()
    assert np.abs(H1 - H0).max() <= 2e-4 * np.abs(H0).max()
    for (s, c, b) in samples:
        Hr = orc.energy(L, J[s], eng.get_spins(s, c, b))
        assert abs(H1[s, c, b] - Hr) <= 2e-5 * abs(Hr)
    eng.close()


@pytest.mark.parametrize("name,chains", [
    ("L16_R24_S64", [(5, 0), (40, 1)]),
    ("L32_R48_S16", [(3, 1)]),
])
def test_fullsize_exchange_sampled(name, chains):
    w, eng, J, B = _engine(name)
    L = w.L[0]
    NT = w.n_replicas[0]
    mode = {"plain": 0, "decimation": 1, "coolheat": 2}[w.exchange]
    eng.sweep(w.n_hb, w.n_or)
    eng.exchange(w.exchange)
    eng.sweep(w.n_hb, w.n_or)
    ref = {}
    for (s, c) in chains:
        st = np.stack([eng.get_spins(s, c, b) for b in range(NT)])
        ch = orc.Chain(L, J[s], B[s], st, copy=c, sample=s, seed=7)
        prop, acc, rt, perm = eng.stats()
        ch.label[:] = perm[s, c]
        ref[(s, c)] = (ch, perm[s, c].copy(), acc[s, c].copy())
    step = eng.step
    H0 = eng.energies()
    eps = np.full(NT - 1, w.eps, np.float32)
    eng.exchange(w.exchange)
    prop, acc, rt, perm = eng.stats()
    H = eng.energies()
    # the logged ln A (and ln det J_C terms) of every pair against the oracle
    # walk that follows the engine's decisions, up to the first re-insertion
    # where float and double may part
    lnA, lnJ = eng.exchange_log()
    errors = {}
    for (s, c), (ch, _, _) in ref.items():
        recs = exchange_walk(w.exchange, L, J[s], B[s], ch.spins, H0[s, c], 7, s, c, step, eps=eps,
                             follow_lnA=lnA[s, c])[0]
        float_tolerances(recs, w.exchange, B[s], L ** 3)
        check_float_walk(errors, name, lnA[s, c], lnJ[s, c], recs, L ** 3)
    print(f"\n{name} exchange log vs oracle walk:", errors[name])
    mismatched = 0
    for (s, c), (ch, perm0, acc0) in ref.items():
        ch.exchange(mode, step, eps=eps)
        got_acc = acc[s, c] - acc0
        if not (perm[s, c] == ch.label).all() or not (got_acc == ch.acc).all():
            mismatched += 1
            continue
        for b in range(NT):
            assert abs(H[s, c, b] - ch.H[b]) <= 1e-4 * abs(ch.H[b])
    # float and double decisions differ only where ln A is within float
    # round-off of ln u; at most one sampled chain may show such a tie
    assert mismatched <= max(0, len(chains) - 1)
    eng.close()


def test_fullsize_uneven_batch_sampled():
    """The uneven batch as bench.py runs it (autotuned paths, per-sample
    overrelaxation counts, plain swap): one heat-bath and one overrelaxation
    sweep checked site by site for replicas of every lattice size, on the
    resident kernel each size uses."""
    w = W.uneven_batch()
    Js = w.couplings()
    Bs = w.betas()
    eng = pt.Engine(list(w.L), Js, Bs, n_copies=2, precision="fp32", seed=7)
    nor = [w.extra["n_or_per_L"][L] for L in w.L]
    eng.autotune(w.n_hb, max(nor))
    choice, ctas = eng.paths()
    assert (choice >= 10).all()                           # every sample resident
    picks = {}
    for s, L in enumerate(w.L):
        picks.setdefault(L, s)
    for L, s in picks.items():
        assert (ctas[s] == 1) == (L <= 16), (L, ctas[s])  # clusters only above L = 16
    eng.sweep_samples(w.n_hb, nor)
    eng.exchange(w.exchange)
    off = np.concatenate([[0], np.cumsum([2 * n for n in w.n_replicas])])
    for kind, (nh, no) in (("hb", (1, 0)), ("or", (0, 1))):
        tags = [(s, c, b) for s in picks.values() for (c, b) in ((0, 0), (1, w.n_replicas[s] - 1))]
        before = {t: eng.get_spins(*t) for t in tags}
        step0 = eng.step
        eng.sweep_samples(nh, [no] * len(w.L))
        for (s, c, b) in tags:
            L, NT = w.L[s], w.n_replicas[s]
            after = eng.get_spins(s, c, b)
            _check_half_sweeps(L, np.asarray(Js[s], np.float64), before[(s, c, b)], after, kind, Bs[s][b], 7, s,
                               c * NT + b, step0)
            assert np.allclose(np.linalg.norm(after, axis=1), 1.0, atol=1e-5)
    H = eng.energies()
    for (s, c, b) in tags:
        L, NT = w.L[s], w.n_replicas[s]
        Hr = orc.energy(L, np.asarray(Js[s], np.float64), eng.get_spins(s, c, b))
        assert abs(H[off[s] + c * NT + b] - Hr) <= 2e-5 * abs(Hr)
    eng.close()


def test_fullsize_L24_coolheat_cluster_exchange_sampled():
    """Cooling/heating at L = 24 in float, the size the paper's second
    protocol runs (10 coupling sets x 27 replicas x 2 copies on the geometric
    ladder, cooling parameter kappa = 0.1): its configurations do not fit one
    SM, so the exchange runs as the cluster kernel (one launch, no heating
    pre-pass), after autotuned sweeps.  Sampled chains: per pair ln A and the
    two ln det J_C terms against the oracle walk within the float bounds,
    decisions equal outside the round-off band, the final configurations to
    1e-5 per component."""
    L, S, NT, seed = 24, 10, 27, 17
    J = np.stack([W.couplings(L, 8000 + 97 * L + k) for k in range(S)])
    B = np.stack([W.geometric_betas(NT)] * S)
    eps = np.stack([(0.1 * np.log(B[s, 1:] / B[s, :-1])).astype(np.float32) for s in range(S)])
    eng = pt.Engine(L, J, B, n_copies=2, precision="fp32", seed=seed)
    eng.set_params(eps=eps)
    eng.autotune(1, 30)
    choice, _ = eng.paths()
    assert (choice >= 10).all()
    for _ in range(3):
        eng.sweep(1, 30)
        eng.exchange("coolheat")
    eng.sweep(1, 30)
    Jd = J.astype(np.float64)
    N = L ** 3
    chains = [(2, 0), (7, 1)]
    H0 = eng.energies()
    step = eng.step
    start = {(s, c): np.stack([eng.get_spins(s, c, b) for b in range(NT)]) for (s, c) in chains}
    perm0 = eng.stats()[3]
    eng.profile(True)
    eng.exchange("coolheat")
    _, launches = eng.profile_read()
    eng.profile(False)
    assert launches["exchange"] == 1  # the cluster kernel, no heating pre-pass
    perm1 = eng.stats()[3]
    lnA, lnJ = eng.exchange_log()
    errors = {}
    n_acc = 0
    for (s, c) in chains:
        recs, sp, Hw, permw = exchange_walk("coolheat", L, Jd[s], B[s], start[(s, c)], H0[s, c], seed, s, c, step,
                                            eps=eps[s], follow_lnA=lnA[s, c])
        float_tolerances(recs, "coolheat", B[s], N)
        assert check_float_walk(errors, "L24", lnA[s, c], lnJ[s, c], recs, N)
        assert (perm1[s, c] == perm0[s, c][permw]).all()
        for b in range(NT):
            d = np.abs(eng.get_spins(s, c, b) - sp[b]).max()
            errors["L24"]["spin"] = max(errors["L24"]["spin"], float(d))
            assert d <= 1e-5, (s, c, b, d)
        n_acc += sum(bool(r["accepted"]) for r in recs)
    print("\nL=24 cluster cooling/heating, float vs oracle:", errors["L24"], "accepted pairs", n_acc)
    assert n_acc > 0
    eng.close()
