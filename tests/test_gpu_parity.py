"""GPU parity of every kernel of the hot path against the FP64 oracle, element
by element, on seeded inputs: initial spins, heat-bath and overrelaxation half
sweeps, energies, overlap, and the three exchanges.  Lattice sizes cover a
single partial tile (L = 4, 6), several tiles with a ragged tail (L = 12) and
full tiles (L = 16); uneven batches mix sizes in one launch.

Tolerances: double precision 1e-12 per spin component (spec bound);
single precision 1e-5 per spin component after one sweep, relative 1e-5 on
energies; integer bookkeeping bit-exact."""
import numpy as np
import pytest

import oracle as orc
from gpu_util import (ambiguous_basis_sites, check_float_walk, exchange_walk, float_tolerances, get_state,
                      make_engine, set_random_state, site_colour)

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1006_4247_gb300 import _build
    _build.build()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("L", [2, 4, 6, 12])
def test_initial_spins(precision, L):
    S, C, NT = 2, 2, 3
    eng, J, B = make_engine(L, S, NT, C, precision, seed=77)
    st = get_state(eng, S, C, NT)
    for s in range(S):
        for c in range(C):
            for b in range(NT):
                ref = orc.init_spins(L, 0, 77, s, c * NT + b)
                assert np.abs(st[s, c, b] - ref).max() <= TOL[precision], (s, c, b)
    eng.close()
    eng, J, B = make_engine(L, S, NT, C, precision, start="ordered")
    assert (get_state(eng, S, C, NT) == np.array([1.0, 0.0, 0.0])).all()
    eng.close()


@pytest.mark.parametrize("L", [2, 4, 6, 12, 16])
def test_energy_and_overlap(L):
    S, C, NT = 2, 2, 3
    for precision in ("fp64", "fp32"):
        eng, J, B = make_engine(L, S, NT, C, precision)
        st = set_random_state(eng, S, C, NT, L, seed=5)
        H = eng.energies()
        Q, chi = eng.overlap()
        for s in range(S):
            for c in range(C):
                for b in range(NT):
                    ref = orc.energy(L, J[s], st[s, c, b])
                    tol = 1e-11 if precision == "fp64" else 2e-5
                    assert abs(H[s, c, b] - ref) <= tol * max(1.0, abs(ref))
            for b in range(NT):
                Qr, chir = orc.overlap(L, st[s, 0, b], st[s, 1, b])
                tol = 1e-10 if precision == "fp64" else 1e-4
                assert np.abs(Q[s, b] - Qr).max() <= tol * max(1.0, np.abs(Qr).max())
                assert abs(chi[s, b] - chir) <= tol * max(1.0, chir)
        eng.close()


def _oracle_sweep(L, J, s, beta, kind, seed, sample, rep_id, step):
    t = s.copy()
    for colour in (0, 1):
        if kind == "hb":
            t = orc.hb_halfsweep(L, J, t, colour, beta, seed, sample, rep_id, step + colour)
        else:
            t = orc.or_halfsweep(L, J, t, colour)
    return t


@pytest.mark.parametrize("L", [2, 4, 6, 12, 16])
@pytest.mark.parametrize("kind", ["hb", "or"])
def test_one_sweep_fp64(L, kind):
    """One sweep (colour 0 then colour 1) from an identical state with identical
    Philox counters matches the oracle to 1e-12."""
    S, C, NT, seed = 2, 2, 3, 21
    eng, J, B = make_engine(L, S, NT, C, "fp64", seed=seed)
    st = set_random_state(eng, S, C, NT, L, seed=9)
    step0 = 1234567
    eng.step = step0
    eng.sweep(1, 0) if kind == "hb" else eng.sweep(0, 1)
    out = get_state(eng, S, C, NT)
    assert eng.step == step0 + 2
    for s in range(S):
        for c in range(C):
            for b in range(NT):
                ref = _oracle_sweep(L, J[s], st[s, c, b], B[s, b], kind, seed, s, c * NT + b, step0)
                assert np.abs(out[s, c, b] - ref).max() <= 1e-12, (s, c, b)
    # the fused energy of the last half sweep equals the oracle's H
    H = eng.energies()
    for s in range(S):
        for c in range(C):
            for b in range(NT):
                ref = orc.energy(L, J[s], out[s, c, b])
                assert abs(H[s, c, b] - ref) <= 1e-11 * max(1, abs(ref))
    eng.close()


@pytest.mark.parametrize("L", [4, 12, 16])
@pytest.mark.parametrize("kind", ["hb", "or"])
def test_one_sweep_fp32(L, kind):
    """Single precision: each half sweep is checked site by site, the second
    one from the engine's own first-half result (the oracle computes every
    site from the same neighbours); where the heat-bath basis orientation is
    ambiguous only the component along S and |s| = 1 are compared."""
    S, C, NT, seed = 1, 2, 3, 23
    eng, J, B = make_engine(L, S, NT, C, "fp32", seed=seed)
    st = set_random_state(eng, S, C, NT, L, seed=19)
    step0 = 99
    eng.step = step0
    eng.sweep(1, 0) if kind == "hb" else eng.sweep(0, 1)
    out = get_state(eng, S, C, NT)
    col = site_colour(L)
    for c in range(C):
        for b in range(NT):
            cur = st[0, c, b].copy()
            for colour in (0, 1):
                if kind == "hb":
                    ref = orc.hb_halfsweep(L, J[0], cur, colour, B[0, b], seed, 0, c * NT + b, step0 + colour)
                    amb = ambiguous_basis_sites(L, J[0], cur, colour)
                else:
                    ref = orc.or_halfsweep(L, J[0], cur, colour)
                    amb = np.zeros(L ** 3, bool)
                m = (col == colour) & ~amb
                assert np.abs(out[0, c, b][m] - ref[m]).max() <= 1e-5, (c, b, colour)
                for x in np.nonzero((col == colour) & amb)[0]:
                    Sx = orc.local_field(L, J[0], cur, x)
                    n = Sx / np.linalg.norm(Sx)
                    assert abs(out[0, c, b][x] @ n - ref[x] @ n) <= 1e-5
                # continue from the engine's half-sweep result
                cur = cur.copy()
                cur[col == colour] = out[0, c, b][col == colour]
            assert np.allclose(np.linalg.norm(out[0, c, b], axis=1), 1.0, atol=1e-6)
    eng.close()


def _oracle_chains(eng_state, J, B, S, C, NT, L, seed):
    chains = []
    for s in range(S):
        for c in range(C):
            chains.append(orc.Chain(L, J[s], B[s], eng_state[s, c], copy=c, sample=s, seed=seed))
    return chains


# Exchange kernels: "auto" runs the staged kernels (the pair in shared memory;
# k_heat_pre + k_exchange_coolheat_smem, k_exchange_decimation_smem) at these
# sizes; "l2:<n>" forces the cluster kernels (k_exchange_coolheat,
# k_exchange_decimation) with n CTAs per chain, the ones float batches with
# L > 20 and double batches with L > 16 run.
EXCHANGE_IMPLS = {"auto": {}, "l2:1": {"PT_EXCHANGE_IMPL": "l2", "PT_EXCHANGE_CLUSTER": "1"},
                  "l2:2": {"PT_EXCHANGE_IMPL": "l2", "PT_EXCHANGE_CLUSTER": "2"},
                  "l2:4": {"PT_EXCHANGE_IMPL": "l2", "PT_EXCHANGE_CLUSTER": "4"}}
EXCHANGE_CASES = [("plain", "auto")] + [(m, i) for m in ("decimation", "coolheat") for i in EXCHANGE_IMPLS]


@pytest.mark.parametrize("mode,impl", EXCHANGE_CASES)
@pytest.mark.parametrize("L", [4, 6, 12])
def test_exchange_fp64(mode, impl, L):
    """One tempering update from identical state: permutation, counters,
    round trips bit-exact; spins (re-inserted or transformed) to 1e-12;
    energies to 1e-11; the logged ln A (and the two ln det J_C terms of
    cooling/heating) of every pair to 1e-9 of the oracle walk's."""
    S, C, NT, seed = 2, 2, 6, 31
    eng, J, B = _engine_env(EXCHANGE_IMPLS[impl], L, S, NT, C, "fp64", seed=seed, bmin=1.8, bmax=2.4)
    st = set_random_state(eng, S, C, NT, L, seed=29)
    chains = _oracle_chains(st, J, B, S, C, NT, L, seed)
    eps = np.full((S, NT - 1), 0.02, np.float32)
    for rnd in range(4):
        step = eng.step
        H0 = eng.energies()
        walks = [exchange_walk(mode, L, J[s], B[s], get_state(eng, S, C, NT)[s, c], H0[s, c], seed, s, c, step,
                               eps=eps[s]) for s in range(S) for c in range(C)]
        eng.exchange(mode, eps if mode == "coolheat" else None)
        for ch in chains:
            ch.exchange({"plain": 0, "decimation": 1, "coolheat": 2}[mode], step, eps=eps[0])
        prop, acc, rt, perm = eng.stats()
        H = eng.energies()
        out = get_state(eng, S, C, NT)
        lnA, lnJ = eng.exchange_log()
        for s in range(S):
            for c in range(C):
                ch = chains[s * C + c]
                assert (perm[s, c] == ch.label).all(), (rnd, s, c)
                assert (prop[s, c] == ch.prop).all() and (acc[s, c] == ch.acc).all()
                assert rt[s, c] == ch.rt_count[0]
                assert np.abs(out[s, c] - ch.spins).max() <= 1e-12
                assert np.abs(H[s, c] - ch.H).max() <= 1e-11 * max(1.0, np.abs(ch.H).max())
                recs = walks[s * C + c][0]
                for i, r in enumerate(recs):
                    assert abs(lnA[s, c, i] - r["lnA"]) <= 1e-9 * max(1.0, abs(r["lnA"])), (rnd, s, c, i)
                    assert abs(lnJ[s, c, i, 0] - r["lnJ1"]) <= 1e-9 * max(1.0, abs(r["lnJ1"]))
                    assert abs(lnJ[s, c, i, 1] - r["lnJ2"]) <= 1e-9 * max(1.0, abs(r["lnJ2"]))
        # move the state on and start the next update from an identical state
        # (the oracle takes the engine's spins; its bookkeeping continues)
        eng.sweep(0, 1)
        new = get_state(eng, S, C, NT)
        for s in range(S):
            for c in range(C):
                ch = chains[s * C + c]
                ch.spins[:] = new[s, c]
                for b in range(NT):
                    ch.H[b] = orc.energy(L, ch.J, ch.spins[b])
    assert sum(int(c.acc.sum()) for c in chains) > 0
    eng.close()


FLOAT_ERRORS = {}


# decimation re-inserts sites by heat bath, where float and double may orient
# a site's basis oppositely (|S_z| < 1e-4 |S|, about one site in 10^4): kept to
# L <= 8 so that the walks rarely part there
FLOAT_WALK_CASES = [(m, i, L) for i in ("auto", "l2:2") for m, Ls in (("decimation", (6, 8)),
                                                                        ("coolheat", (6, 8, 16))) for L in Ls]


@pytest.mark.parametrize("mode,impl,L", FLOAT_WALK_CASES)
def test_exchange_fp32_elementwise(mode, impl, L):
    """Single precision decimation and cooling/heating, staged and cluster
    kernels, one tempering update from an identical state: per pair ln A and
    ln det J_C(s1), ln det J_C(C^-1 s2) against the oracle walk within the
    bounds of gpu_util; decisions equal outside the round-off band of ln u
    (the walk follows the engine inside it); the final configurations
    (re-inserted, cooled and heated) to 1e-5 per component, the energies to
    2e-5, the permutation exactly."""
    S, C, NT, seed = 2, 2, 6, 43
    eng, J, B = _engine_env(EXCHANGE_IMPLS[impl], L, S, NT, C, "fp32", seed=seed, bmin=1.8, bmax=2.4)
    set_random_state(eng, S, C, NT, L, seed=47)
    N = L ** 3
    # a cooling parameter near the acceptance optimum of this ladder (kappa ~ 0.1)
    eps = np.full((S, NT - 1), 0.1 * np.log(B[0, 1] / B[0, 0]), np.float32)
    name = f"{mode}/{impl}"
    compared = 0
    for rnd in range(2):
        step = eng.step
        H0 = eng.energies()
        state = get_state(eng, S, C, NT)
        perm0 = eng.stats()[3]
        eng.exchange(mode, eps if mode == "coolheat" else None)
        perm1 = eng.stats()[3]
        lnA, lnJ = eng.exchange_log()
        out = get_state(eng, S, C, NT)
        H = eng.energies()
        for s in range(S):
            for c in range(C):
                recs, sp, Hw, permw = exchange_walk(mode, L, J[s], B[s], state[s, c], H0[s, c], seed, s, c, step,
                                                    eps=eps[s], follow_lnA=lnA[s, c])
                float_tolerances(recs, mode, B[s], N)
                if not check_float_walk(FLOAT_ERRORS, name, lnA[s, c], lnJ[s, c], recs, N):
                    continue
                assert (perm1[s, c] == perm0[s, c][permw]).all(), (name, s, c)
                d = float(np.abs(out[s, c] - sp).max())
                FLOAT_ERRORS[name]["spin"] = max(FLOAT_ERRORS[name]["spin"], d)
                assert d <= 1e-5, (name, s, c, d)
                assert np.abs(H[s, c] - Hw).max() <= 2e-5 * np.abs(Hw).max()
                compared += 1
        eng.sweep(0, 1)
    assert compared >= 2 * S * C - 2
    print(f"\nfloat exchange errors vs oracle ({name}, L={L}):", FLOAT_ERRORS[name])
    eng.close()


@pytest.mark.parametrize("mode", ["plain", "decimation", "coolheat"])
def test_exchange_fp32_statistics_match_decisions(mode):
    """Single precision exchange from an identical state: decisions agree with
    the oracle's except where |ln A| is within float round-off of ln u."""
    L, S, C, NT, seed = 6, 4, 2, 6, 41
    eng, J, B = make_engine(L, S, NT, C, "fp32", seed=seed, bmin=1.8, bmax=2.4)
    st = set_random_state(eng, S, C, NT, L, seed=39)
    chains = _oracle_chains(st, J, B, S, C, NT, L, seed)
    eps = np.full((S, NT - 1), 0.02, np.float32)
    step = eng.step
    eng.exchange(mode, eps if mode == "coolheat" else None)
    for ch in chains:
        ch.exchange({"plain": 0, "decimation": 1, "coolheat": 2}[mode], step, eps=eps[0])
    prop, acc, rt, perm = eng.stats()
    agree = sum(int((perm[s, c] == chains[s * C + c].label).all()) for s in range(S) for c in range(C))
    assert agree >= S * C - 1
    eng.close()


def test_uneven_batch_parity():
    """Samples of different L and replica counts in one engine (one launch per
    half sweep) match the oracle sample by sample."""
    from paper_1006_4247_gb300 import pt
    from paper_1006_4247_gb300 import workloads as W
    Ls = [4, 6, 8, 2, 12]
    NTs = [3, 5, 2, 4, 3]
    Js = [W.couplings(L, 500 + i) for i, L in enumerate(Ls)]
    Bs = [W.linear_betas(n, 0.7, 1.9) for n in NTs]
    seed = 51
    eng = pt.Engine(Ls, Js, Bs, n_copies=2, precision="fp64", seed=seed)
    for s, L in enumerate(Ls):
        for c in range(2):
            for b in range(NTs[s]):
                ref = orc.init_spins(L, 0, seed, s, c * NTs[s] + b)
                assert np.abs(eng.get_spins(s, c, b) - ref).max() <= 1e-12
    before = [[[eng.get_spins(s, c, b) for b in range(NTs[s])] for c in range(2)] for s in range(len(Ls))]
    step0 = eng.step
    eng.sweep(1, 1)
    for s, L in enumerate(Ls):
        J = Js[s].astype(np.float64)
        for c in range(2):
            for b in range(NTs[s]):
                ref = _oracle_sweep(L, J, before[s][c][b], Bs[s][b], "hb", seed, s, c * NTs[s] + b, step0)
                ref = _oracle_sweep(L, J, ref, Bs[s][b], "or", seed, s, 0, 0)
                assert np.abs(eng.get_spins(s, c, b) - ref).max() <= 1e-12, (s, c, b)
    H, Q, chi = eng.measure()
    off = 0
    qoff = 0
    for s, L in enumerate(Ls):
        J = Js[s].astype(np.float64)
        for c in range(2):
            for b in range(NTs[s]):
                ref = orc.energy(L, J, eng.get_spins(s, c, b))
                assert abs(H[off] - ref) <= 1e-11 * max(1, abs(ref))
                off += 1
        for b in range(NTs[s]):
            Qr, chir = orc.overlap(L, eng.get_spins(s, 0, b), eng.get_spins(s, 1, b))
            assert abs(chi[qoff] - chir) <= 1e-10 * max(1, chir)
            qoff += 1
    eng.close()


@pytest.mark.parametrize("L,n_hb,n_or", [(8, 1, 3), (16, 1, 3), (24, 1, 3), (32, 1, 3),
                                         (16, 2, 1), (16, 0, 2), (32, 2, 1), (32, 0, 2)])
def test_resident_and_streaming_paths_fp64(L, n_hb, n_or):
    """A block of n_hb heat-bath + n_or overrelaxation sweeps through the
    shared-memory resident kernel and through the streaming half sweeps gives
    the oracle's configuration (1e-12 per sweep) and the same energies.  With
    a heat-bath sweep first the resident block does not load colour 0 (the
    first half sweep redraws it); without one it loads the whole replica."""
    S, C, NT, seed = 2, 2, 3, 61
    res = {}
    for policy in ("resident", "streaming"):
        eng, J, B = make_engine(L, S, NT, C, "fp64", seed=seed)
        eng.set_policy(policy)
        st = set_random_state(eng, S, C, NT, L, seed=7)
        step0 = 4242
        eng.step = step0
        eng.profile(True)
        eng.sweep(n_hb, n_or)
        ms, n = eng.profile_read()
        assert (n["resident"] > 0) == (policy == "resident")
        out = get_state(eng, S, C, NT)
        H = eng.energies()
        for s in range(S):
            for c in range(C):
                for b in range(NT):
                    ref = st[s, c, b]
                    for k in range(n_hb):
                        ref = _oracle_sweep(L, J[s], ref, B[s, b], "hb", seed, s, c * NT + b, step0 + 2 * k)
                    for _ in range(n_or):
                        ref = _oracle_sweep(L, J[s], ref, B[s, b], "or", seed, s, 0, 0)
                    # several sweeps: 1e-12 per sweep grows through the chaotic updates
                    assert np.abs(out[s, c, b] - ref).max() <= 1e-11, (policy, s, c, b)
                    Hr = orc.energy(L, J[s], out[s, c, b])
                    assert abs(H[s, c, b] - Hr) <= 1e-11 * max(1, abs(Hr))
        assert eng.step == step0 + 2 * (n_hb + n_or)
        res[policy] = out
        eng.close()
    assert np.abs(res["resident"] - res["streaming"]).max() <= 1e-14


@pytest.mark.parametrize("L", [16, 24, 32])
def test_resident_and_streaming_paths_fp32(L):
    """L = 16 runs in one CTA per replica, L = 24 and 32 in clusters of 2 and
    4 CTAs (slabs of z planes)."""
    S, C, NT, seed = 2, 2, 3, 63
    res = {}
    for policy in ("resident", "streaming"):
        eng, J, B = make_engine(L, S, NT, C, "fp32", seed=seed)
        eng.set_policy(policy)
        set_random_state(eng, S, C, NT, L, seed=8)
        eng.sweep(1, 2)
        res[policy] = (get_state(eng, S, C, NT), eng.energies())
        eng.close()
    assert np.abs(res["resident"][0] - res["streaming"][0]).max() <= 1e-6
    assert np.abs(res["resident"][1] - res["streaming"][1]).max() <= 1e-3


@pytest.mark.parametrize("L,precision,cs", [(24, "fp32", 4), (32, "fp32", 8), (24, "fp64", 8)])
def test_narrow_cluster_path_vs_oracle(L, precision, cs):
    """Clusters of 512-thread CTAs (two per SM; L = 24 in slabs of 6 planes
    and L = 32 of 4 in float, L = 24 of 3 in double): one heat-bath and two
    overrelaxation sweeps against the streaming half sweeps and, in double,
    against the oracle site by site."""
    S, C, NT, seed = 2, 2, 2, 65
    eng, J, B = _engine_env({"PT_CL_NARROW": "1"}, L, S, NT, C, precision, seed=seed)
    choice, ctas = eng.paths()
    assert (choice // 10 == 2).all() and (ctas == cs).all()
    st = set_random_state(eng, S, C, NT, L, seed=9)
    step0 = 777
    eng.step = step0
    eng.sweep(1, 2)
    out = get_state(eng, S, C, NT)
    H = eng.energies()
    ref_eng, _, _ = make_engine(L, S, NT, C, precision, seed=seed)
    ref_eng.set_policy("streaming")
    for s in range(S):
        for c in range(C):
            for b in range(NT):
                ref_eng.set_spins(s, c, b, st[s, c, b])
    ref_eng.step = step0
    ref_eng.sweep(1, 2)
    assert np.abs(get_state(ref_eng, S, C, NT) - out).max() <= (1e-14 if precision == "fp64" else 1e-6)
    ref_eng.close()
    if precision == "fp64":  # float: the streaming path above is itself checked against the oracle
        for s in range(S):
            for c in range(C):
                for b in range(NT):
                    ref = _oracle_sweep(L, J[s], st[s, c, b], B[s, b], "hb", seed, s, c * NT + b, step0)
                    for _ in range(2):
                        ref = _oracle_sweep(L, J[s], ref, B[s, b], "or", seed, s, 0, 0)
                    assert np.abs(out[s, c, b] - ref).max() <= 1e-11, (s, c, b)
                    Hr = orc.energy(L, J[s], out[s, c, b])
                    assert abs(H[s, c, b] - Hr) <= 1e-11 * max(1, abs(Hr))
    eng.close()


def test_policy_errors():
    from paper_1006_4247_gb300 import pt
    eng, J, B = make_engine(2, 1, 3, 2, "fp32")  # rows of one site: no resident kernel
    with pytest.raises(pt.PtError) as ei:
        eng.set_policy("resident")
    assert ei.value.status == pt.PT_ERR_STATE
    eng.set_policy("streaming")
    eng.close()


def _engine_env(env, *args, **kw):
    import os
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        return make_engine(*args, **kw)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.mark.parametrize("L", [8, 16, 24, 32])
def test_bulk_copy_half_sweep_matches_plain_loads(L):
    """The overrelaxation half sweep with TMA-staged slabs gives the same
    spins as the one with plain vector loads (streaming policy)."""
    S, C, NT = 2, 2, 3
    out = {}
    for tma in ("1", "0"):
        eng, J, B = _engine_env({"PT_TMA": tma}, L, S, NT, C, "fp32", seed=3)
        eng.set_policy("streaming")
        set_random_state(eng, S, C, NT, L, seed=13)
        eng.profile(True)
        eng.sweep(0, 3)
        out[tma] = (get_state(eng, S, C, NT), eng.energies())
        eng.close()
    assert np.abs(out["1"][0] - out["0"][0]).max() <= 1e-6
    assert np.abs(out["1"][1] - out["0"][1]).max() <= 1e-3


@pytest.mark.parametrize("L", [16, 32])
def test_bulk_copy_half_sweep_vs_oracle(L):
    """Two overrelaxation sweeps through the TMA path, checked half sweep by
    half sweep against the oracle."""
    S, C, NT = 1, 2, 2
    eng, J, B = _engine_env({"PT_TMA": "1"}, L, S, NT, C, "fp32", seed=5)
    eng.set_policy("streaming")
    st = set_random_state(eng, S, C, NT, L, seed=15)
    eng.sweep(0, 1)  # colour 0 through the bulk-copy kernel, colour 1 with the energy
    out = get_state(eng, S, C, NT)
    col = site_colour(L)
    for c in range(C):
        for b in range(NT):
            cur = st[0, c, b].copy()
            for colour in (0, 1):
                ref = orc.or_halfsweep(L, J[0], cur, colour)
                m = col == colour
                assert np.abs(out[0, c, b][m] - ref[m]).max() <= 1e-5
                cur = cur.copy()
                cur[m] = out[0, c, b][m]
    eng.close()
