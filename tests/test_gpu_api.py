"""GPU checks of the C ABI around the hot path: exact checkpoint/resume,
error statuses, the PyTorch allocator hook, asynchronous device-side
measurement and the per-kernel profiler."""
import os

import numpy as np
import pytest

from gpu_util import get_state, make_engine
from paper_1006_4247_gb300 import pt
from paper_1006_4247_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1006_4247_gb300 import _build
    _build.build()


def _cycles(eng, n, mode, eps=None):
    for _ in range(n):
        eng.sweep(1, 2)
        eng.exchange(mode, eps)


@pytest.mark.parametrize("mode", ["plain", "decimation", "coolheat"])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_checkpoint_resume_is_exact(tmp_path, mode, precision):
    """k cycles, save, k cycles == load into a fresh engine, k cycles."""
    L, S, NT = 8, 2, 4
    eps = np.full(S * (NT - 1), 0.03, np.float32)
    a, J, B = make_engine(L, S, NT, 2, precision, seed=17)
    a.set_params(eps=eps)
    _cycles(a, 3, mode)
    f = str(tmp_path / "ck.bin")
    a.save(f)
    _cycles(a, 3, mode)
    ref_state, ref_stats, ref_H = get_state(a, S, 2, NT), a.stats(), a.energies()
    b, _, _ = make_engine(L, S, NT, 2, precision, seed=17)
    b.load(f)
    _cycles(b, 3, mode)
    assert (get_state(b, S, 2, NT) == ref_state).all()
    for x, y in zip(b.stats(), ref_stats):
        assert (x == y).all()
    assert (b.energies() == ref_H).all()
    assert a.step == b.step
    a.close()
    b.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_set_spins_normalises_and_rejects_zero(precision):
    """Spins enter the engine as unit vectors (the updates' renormalisation
    only corrects rounding): pt_set_spins scales spins of other lengths to
    unit length, keeps unit ones as given, and refuses a zero spin, leaving
    the stored configuration unchanged."""
    L = 4
    eng, J, B = make_engine(L, 1, 3, 2, precision)
    v = W.random_spins(L, 5) * np.linspace(0.5, 3.0, L ** 3)[:, None]
    eng.set_spins(0, 1, 2, v)
    got = eng.get_spins(0, 1, 2)
    tol = 1e-15 if precision == "fp64" else 1e-7
    assert np.abs(np.linalg.norm(got, axis=1) - 1.0).max() <= 2 * tol
    assert np.abs(got - v / np.linalg.norm(v, axis=1, keepdims=True)).max() <= 2 * tol
    eng.set_spins(0, 1, 2, got)  # unit to float accuracy: stored bit for bit
    assert (eng.get_spins(0, 1, 2) == got).all()
    bad = got.copy()
    bad[7] = 0.0
    with pytest.raises(pt.PtError) as ei:
        eng.set_spins(0, 1, 2, bad)
    assert ei.value.status == pt.PT_ERR_ARG and "zero" in str(ei.value)
    assert (eng.get_spins(0, 1, 2) == got).all()
    eng.close()


def test_exchange_log_and_smem_probe():
    """pt_get_exchange_log is zero before the first tempering update and holds
    every pair's ln A afterwards (the standard swap: (b2 - b1)(H2 - H1) of the
    energies before the update, no Jacobian terms); pt_smem_bandwidth reports
    a rate between 10 and 100 TB/s (GB300: about 40), up to 256 B per clock per
    SM, and the clock it ran at."""
    eng, J, B = make_engine(8, 2, 4, 2, "fp32")
    lnA, lnJ = eng.exchange_log()
    assert lnA.shape == (2, 2, 3) and lnJ.shape == (2, 2, 3, 2)
    assert (lnA == 0).all() and (lnJ == 0).all()
    H0 = eng.energies()
    eng.exchange("plain")
    lnA, lnJ = eng.exchange_log()
    assert (lnJ == 0).all()
    # pair 0 of each chain sees the energies before the update
    ref = (B[:, 1] - B[:, 0])[:, None] * (H0[:, :, 1] - H0[:, :, 0])
    assert np.allclose(lnA[:, :, 0], ref, rtol=1e-12, atol=1e-12)
    eng.close()
    bps, bpc, mhz = pt.pt_smem_bandwidth()
    assert 10e12 < bps < 100e12 and 0 < bpc <= 256 and 500 < mhz < 3000, (bps, bpc, mhz)


def test_error_statuses():
    eng, J, B = make_engine(4, 1, 3, 2, "fp32")
    with pytest.raises(pt.PtError) as ei:
        eng.exchange("coolheat", np.full(2, 10.0, np.float32))  # eps * max sum|J| >= 1
    assert ei.value.status == pt.PT_ERR_EPS
    with pytest.raises(pt.PtError) as ei:
        eng.exchange("coolheat", np.full(2, -0.1, np.float32))
    assert ei.value.status == pt.PT_ERR_EPS
    with pytest.raises(pt.PtError) as ei:
        eng.set_params(betas=np.array([1.0, 0.5, 2.0]))
    assert ei.value.status == pt.PT_ERR_ARG
    with pytest.raises(pt.PtError) as ei:
        eng.get_spins(0, 2, 0)
    assert ei.value.status == pt.PT_ERR_ARG
    with pytest.raises(pt.PtError) as ei:
        pt.pt_exchange(eng.h, 7)
    assert ei.value.status == pt.PT_ERR_ARG
    # the handle is still usable after errors
    eng.sweep(1, 1)
    eng.exchange("plain")
    assert np.isfinite(eng.energies()).all()
    eng.close()
    one, _, _ = make_engine(4, 1, 3, 1, "fp32")
    with pytest.raises(pt.PtError) as ei:
        one.overlap()
    assert ei.value.status == pt.PT_ERR_STATE
    one.close()


def test_load_rejects_other_shapes(tmp_path):
    a, _, _ = make_engine(4, 1, 3, 2, "fp32")
    f = str(tmp_path / "a.bin")
    a.save(f)
    b, _, _ = make_engine(4, 1, 4, 2, "fp32")
    with pytest.raises(pt.PtError) as ei:
        b.load(f)
    assert ei.value.status == pt.PT_ERR_STATE
    with open(str(tmp_path / "junk.bin"), "wb") as fh:
        fh.write(b"not a checkpoint")
    with pytest.raises(pt.PtError):
        b.load(str(tmp_path / "junk.bin"))
    a.close()
    b.close()


def test_torch_allocator_and_stream():
    torch = pytest.importorskip("torch")
    L, S, NT = 8, 2, 3
    J = np.stack([W.couplings(L, 5 + s) for s in range(S)])
    B = np.stack([W.linear_betas(NT, 1.0, 2.0)] * S)
    before = torch.cuda.memory_allocated()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a = pt.Engine(L, J, B, seed=4, use_torch_allocator=True)
        assert torch.cuda.memory_allocated() > before
        a.sweep(1, 2)
        a.exchange("decimation")
        Ha = a.energies()
    b = pt.Engine(L, J, B, seed=4)
    b.sweep(1, 2)
    b.exchange("decimation")
    assert (b.energies() == Ha).all()
    a.close()
    b.close()
    assert torch.cuda.memory_allocated() <= before + (1 << 20)


def test_measure_device_and_profiler():
    torch = pytest.importorskip("torch")
    eng, J, B = make_engine(8, 2, 3, 2, "fp32")
    eng.profile(True)
    eng.sweep(1, 1)
    eng.exchange("plain")
    dH = torch.zeros(2 * 2 * 3, dtype=torch.float64, device="cuda")
    dX = torch.zeros(2 * 3, dtype=torch.float64, device="cuda")
    pt.pt_measure_device(eng.h, dH.data_ptr(), None, dX.data_ptr())
    torch.cuda.synchronize()
    ms, n = eng.profile_read()
    H = eng.energies().ravel()
    Q, chi = eng.overlap()
    assert np.allclose(dH.cpu().numpy(), H)
    assert np.allclose(dX.cpu().numpy(), chi.ravel())
    assert n["exchange"] == 1 and n["measure"] == 1 and sum(n.values()) >= 4
    assert all(v >= 0 for v in ms.values())
    eng.close()


def test_bounded_wait_gives_up_and_handle_stays_usable(monkeypatch):
    """The bulk-copy half sweep's mbarrier wait runs out (one stage's copies
    are never issued): the next synchronising call returns PT_ERR_TIMEOUT once,
    the spins stay unit vectors, and the same handle then sweeps exactly like
    a handle that never failed."""
    from gpu_util import set_random_state
    L, S, NT, C = 16, 1, 3, 2
    monkeypatch.setenv("PT_TMA", "1")
    eng, J, B = make_engine(L, S, NT, C, "fp32", seed=9)
    eng.set_policy("streaming")
    monkeypatch.delenv("PT_TMA")
    ref, _, _ = make_engine(L, S, NT, C, "fp32", seed=9)
    ref.set_policy("streaming")
    eng.set_wait_limit(1024, inject=True)
    eng.sweep(0, 1)  # colour 0 through the bulk-copy kernel, colour 1 with the energy
    with pytest.raises(pt.PtError) as ei:
        eng.energies()
    assert ei.value.status == pt.PT_ERR_TIMEOUT
    s = get_state(eng, S, C, NT)
    assert np.abs(np.linalg.norm(s, axis=-1) - 1.0).max() < 1e-5
    eng.set_wait_limit(0, inject=False)
    out = []
    for e in (eng, ref):
        set_random_state(e, S, C, NT, L, seed=19)
        e.sweep(0, 3)
        out.append((get_state(e, S, C, NT), e.energies()))
    assert np.abs(out[0][0] - out[1][0]).max() <= 1e-6
    assert np.abs(out[0][1] - out[1][1]).max() <= 1e-3
    eng.close()
    ref.close()
    plain, _, _ = make_engine(8, 1, 3, 2, "fp32")
    plain.set_policy("streaming")
    with pytest.raises(pt.PtError) as ei:
        plain.set_wait_limit(16, inject=True)  # streaming without bulk copies: nothing to fault
    assert ei.value.status == pt.PT_ERR_STATE
    plain.close()


@pytest.mark.parametrize("L", [16, 32])
def test_resident_wait_gives_up_and_leaves_replica(L):
    """The resident block's bulk-copy wait runs out for CTA 0 (L = 16: one CTA
    per replica) or for the first cluster (L = 32): the next synchronising call
    returns PT_ERR_TIMEOUT once, the replica whose copies never came is left as
    it was (the whole cluster skips its block), every spin stays a unit
    vector, and the handle then sweeps exactly like one that never failed."""
    from gpu_util import set_random_state
    S, NT, C = 1, 2, 2
    eng, J, B = make_engine(L, S, NT, C, "fp32", seed=5)
    eng.set_policy("resident")
    ref, _, _ = make_engine(L, S, NT, C, "fp32", seed=5)
    ref.set_policy("resident")
    before = get_state(eng, S, C, NT)
    eng.set_wait_limit(1024, inject=True)
    eng.sweep(1, 2)
    ref.sweep(1, 2)  # the same step count on both handles
    with pytest.raises(pt.PtError) as ei:
        eng.energies()
    assert ei.value.status == pt.PT_ERR_TIMEOUT
    after = get_state(eng, S, C, NT)
    assert np.array_equal(after[0, 0, 0], before[0, 0, 0])  # the first replica: CTA 0's
    assert np.abs(np.linalg.norm(after, axis=-1) - 1.0).max() < 1e-5
    eng.set_wait_limit(0, inject=False)
    out = []
    for e in (eng, ref):
        set_random_state(e, S, C, NT, L, seed=23)
        e.sweep(1, 2)
        out.append((get_state(e, S, C, NT), e.energies()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    eng.close()
    ref.close()


def test_set_paths_and_cached_autotune(tmp_path):
    """pt_set_paths applies path codes (and refuses codes a sample cannot
    run, changing nothing); the autotuner's result is stored in a cache file
    and applied from it the next time, without timing again."""
    eng, J, B = make_engine(32, 2, 3, 2, "fp32", seed=3)
    eng.set_paths([24, 24])
    choice, ctas = eng.paths()
    assert list(choice) == [24, 24] and list(ctas) == [8, 8]
    eng.set_paths([14, 4])
    choice, ctas = eng.paths()
    assert list(choice) == [14, 4] and list(ctas) == [4, 0]
    for bad, status in (([3, 4], pt.PT_ERR_ARG), ([34, 4], pt.PT_ERR_ARG), ([11, 4], pt.PT_ERR_STATE)):
        with pytest.raises(pt.PtError) as ei:
            eng.set_paths(bad)
        assert ei.value.status == status
        assert list(eng.paths()[0]) == [14, 4]
    f = str(tmp_path / "tune.json")
    c1, b1 = eng.autotune(1, 2, cache=f)
    assert os.path.exists(f)
    eng.set_paths([4, 4])
    c2, b2 = eng.autotune(1, 2, cache=f)  # from the file
    assert (c2 == c1).all() and (b2 == b1).all()
    assert (eng.paths()[0] == c1).all()
    eng.sweep(1, 1)
    assert np.isfinite(eng.energies()).all()
    eng.close()
