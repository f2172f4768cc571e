"""Uneven batches, per-sample sweep counts, captured update cycles and the
autotuner: each must leave the chain exactly as the plain calls do.

Uneven batch: samples of L = 4, 6, 8, 12, 16, 24 (and replica counts 2..5) in
one engine.  With the default policy, in double precision, L = 4, 8, 12, 16
run one replica per CTA in shared memory, L = 24 one replica per cluster of 4
CTAs (slabs of z planes), and L = 6 (odd row length) in streaming half
sweeps, all inside the same pt_sweep call."""
import numpy as np
import pytest

import oracle as orc
from paper_1006_4247_gb300 import pt
from paper_1006_4247_gb300 import workloads as W

pytestmark = pytest.mark.gpu

LS = [4, 6, 8, 12, 16, 24]
NTS = [3, 2, 4, 3, 2, 5]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1006_4247_gb300 import _build
    _build.build()


def _uneven(precision="fp64", seed=61, stream=None):
    Js = [W.couplings(L, 700 + i) for i, L in enumerate(LS)]
    Bs = [W.linear_betas(n, 0.8, 2.2) for n in NTS]
    eng = pt.Engine(LS, Js, Bs, n_copies=2, precision=precision, seed=seed, stream=stream)
    return eng, [j.astype(np.float64) for j in Js], Bs


def _state(eng):
    return [np.stack([np.stack([eng.get_spins(s, c, b) for b in range(NTS[s])]) for c in range(2)])
            for s in range(len(LS))]


def _oracle_block(L, J, s0, beta, n_hb, n_or, seed, sample, rep_id, step):
    t = s0.copy()
    k = 0
    for _ in range(n_hb):
        for colour in (0, 1):
            t = orc.hb_halfsweep(L, J, t, colour, beta, seed, sample, rep_id, step + k)
            k += 1
    for _ in range(n_or):
        for colour in (0, 1):
            t = orc.or_halfsweep(L, J, t, colour)
    return t


def test_uneven_batch_mixed_paths_vs_oracle():
    eng, Js, Bs = _uneven()
    eng.profile(True)
    before = _state(eng)
    step = eng.step
    n_or = [1, 1, 2, 2, 3, 3]                              # per-sample counts (<= 4 sweeps)
    eng.sweep_samples(1, n_or)
    ms, n = eng.profile_read()
    assert n["resident"] >= 2 and n["hb"] >= 1            # one-CTA and cluster groups, and streaming
    assert eng.step == step + 2 * (1 + max(n_or))
    after = _state(eng)
    H = eng.measure()[0]
    off = 0
    for s, L in enumerate(LS):
        for c in range(2):
            for b in range(NTS[s]):
                ref = _oracle_block(L, Js[s], before[s][c, b], Bs[s][b], 1, n_or[s], 61, s, c * NTS[s] + b, step)
                assert np.abs(after[s][c, b] - ref).max() <= 1e-11, (L, c, b)
                Hr = orc.energy(L, Js[s], after[s][c, b])
                assert abs(H[off] - Hr) <= 1e-10 * max(1, abs(Hr))
                off += 1
    eng.close()


def _run_plain(eng, n, mode, n_or_s=None, measure=True):
    for _ in range(n):
        if n_or_s is None:
            eng.sweep(1, 2)
        else:
            eng.sweep_samples(1, n_or_s)
        eng.exchange(mode)
        if measure:
            eng.measure_device()


@pytest.mark.parametrize("mode", ["plain", "decimation", "coolheat"])
def test_captured_cycles_equal_plain_calls(mode):
    torch = pytest.importorskip("torch")
    st = torch.cuda.Stream()
    n_or_s = [2, 1, 3, 2, 1, 2]
    a, _, _ = _uneven("fp32", seed=5, stream=st.cuda_stream)
    b, _, _ = _uneven("fp32", seed=5, stream=st.cuda_stream)
    eps = np.concatenate([np.full(n - 1, 0.01, np.float32) for n in NTS])
    a.set_params(eps=eps)
    b.set_params(eps=eps)
    a.cycles(4, 1, 0, mode, measure=True, n_or_samples=n_or_s)   # captured graph, replayed 4 times
    a.cycles(3, 1, 0, mode, measure=True, n_or_samples=n_or_s)   # same graph, 3 more
    _run_plain(b, 7, mode, n_or_s)
    for x, y in zip(_state(a), _state(b)):
        assert (x == y).all()
    for x, y in zip(a.stats(), b.stats()):
        assert (x == y).all()
    ma, mb = a.measure(), b.measure()
    for x, y in zip(ma, mb):
        assert (x == y).all()
    assert a.step == b.step
    a.close()
    b.close()


def test_autotune_restores_state_and_keeps_the_chain():
    """After pt_autotune the state is the one before it, and the chain that
    follows agrees with an untuned twin (paths differ only in rounding)."""
    a, _, _ = _uneven("fp64", seed=9)
    b, _, _ = _uneven("fp64", seed=9)
    s0, step0 = _state(a), a.step
    choice, best = a.autotune(1, 2)
    assert len(choice) == len(LS) and (best > 0).all()
    assert all(((c % 10) in (1, 2, 4)) for c in choice)
    for x, y in zip(_state(a), s0):
        assert (x == y).all()
    assert a.step == step0
    _run_plain(a, 2, "decimation", measure=False)
    _run_plain(b, 2, "decimation", measure=False)
    for x, y in zip(_state(a), _state(b)):
        assert np.abs(x - y).max() <= 1e-10
    a.close()
    b.close()
