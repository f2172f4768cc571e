"""The allocation-free energy entry point, pt_energy_noalloc.

It serves callers that cannot let a library call cudaMalloc (a framework's
memory pool that accounts for every device byte, or a loop that forbids
allocation after start-up).  Its partial sums live in a fixed array inside the
library; the caller passes the configurations, the couplings and the output.
Checked here through the C ABI, on two calls in a row so that the second call
cannot profit from what the first one left in the shared array, against the
engine's own energies (pt_measure) and against the FP64 oracle's H computed
configuration by configuration; sizes cover one block per configuration
(L = 4), several blocks with a ragged last one (L = 16: 2 blocks of 2048
sites; L = 32: 16 blocks) and odd L (natural site order has no checkerboard,
so L = 5 is valid here although the engine rejects it).  This file is
collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-11, "fp32": 2e-5}  # relative, as for the engine's energy reduction


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1006_4247_gb300 import _build
    _build.build()
    return torch


def _engine(L, S, NT, precision, seed):
    from paper_1006_4247_gb300 import pt
    from paper_1006_4247_gb300 import workloads as W
    J = np.stack([W.couplings(L, 900 + s) for s in range(S)])
    B = np.stack([W.linear_betas(NT, 0.5, 2.0) for _ in range(S)])
    return pt.Engine(L, J, B, n_copies=2, precision=precision, seed=seed), J


def _noalloc_energies(torch, eng, J, L, S, NT, precision):
    """Energies of every configuration of `eng`, sample by sample, through
    pt_energy_noalloc on torch-owned device buffers."""
    from paper_1006_4247_gb300 import pt
    dt = torch.float64 if precision == "fp64" else torch.float32
    out = np.zeros((S, 2, NT))
    for s in range(S):
        cfg = np.stack([eng.get_spins(s, c, b) for c in range(2) for b in range(NT)])
        d_spins = torch.tensor(cfg, dtype=dt, device="cuda").contiguous()
        d_J = torch.tensor(J[s], dtype=torch.float32, device="cuda").contiguous()
        d_H = torch.full((2 * NT,), float("nan"), dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream()
        pt.pt_energy_noalloc(d_spins.data_ptr(), precision, L, 2 * NT, d_J.data_ptr(),
                             d_H.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        out[s] = d_H.cpu().numpy().reshape(2, NT)
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("L", [4, 16, 32])
def test_noalloc_energy_matches_engine_twice(torch_cuda, precision, L):
    import oracle as orc
    torch = torch_cuda
    S, NT = 2, 3
    eng, J = _engine(L, S, NT, precision, seed=5)
    for call in range(2):
        ref = eng.energies()
        got = _noalloc_energies(torch, eng, J, L, S, NT, precision)
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= TOL[precision] * max(1.0, np.abs(ref).max()), call
        for s in range(S):
            for c in range(2):
                for b in range(NT):
                    Hr = orc.energy(L, J[s].astype(np.float64), eng.get_spins(s, c, b))
                    assert abs(got[s, c, b] - Hr) <= TOL[precision] * max(1.0, abs(Hr)), (call, s, c, b)
        eng.sweep(1, 1)  # new configurations for the second call
    eng.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("L", [3, 5])
def test_noalloc_energy_odd_L_against_oracle_twice(torch_cuda, precision, L):
    """Odd L, which only this entry point accepts: random unit spins from the
    seeded generator, H against the oracle on two calls in a row."""
    import oracle as orc
    from paper_1006_4247_gb300 import pt
    from paper_1006_4247_gb300 import workloads as W
    torch = torch_cuda
    dt = torch.float64 if precision == "fp64" else torch.float32
    J = W.couplings(L, 40 + L)
    d_J = torch.tensor(J, dtype=torch.float32, device="cuda").contiguous()
    for call in range(2):
        cfg = W.random_spins(L, 70 + 10 * call + L, count=5)
        if precision == "fp32":
            cfg = cfg.astype(np.float32).astype(np.float64)  # what the kernel reads
        d_spins = torch.tensor(cfg, dtype=dt, device="cuda").contiguous()
        d_H = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream()
        pt.pt_energy_noalloc(d_spins.data_ptr(), precision, L, 5, d_J.data_ptr(), d_H.data_ptr(),
                             stream.cuda_stream)
        stream.synchronize()
        got = d_H.cpu().numpy()
        for k in range(5):
            Hr = orc.energy(L, J.astype(np.float64), cfg[k])
            assert abs(got[k] - Hr) <= TOL[precision] * max(1.0, abs(Hr)), (call, k)


def test_noalloc_rejects_oversize_and_bad_arguments(torch_cuda):
    torch = torch_cuda
    from paper_1006_4247_gb300 import pt
    L = 32  # 16 partial sums per configuration: at most 4096 configurations
    d_J = torch.zeros(3 * L ** 3, dtype=torch.float32, device="cuda")
    d_H = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(pt.PtError) as ei:
        pt.pt_energy_noalloc(d_J.data_ptr(), "fp32", L, 4097, d_J.data_ptr(), d_H.data_ptr())
    assert ei.value.status == pt.PT_ERR_ARG and "4096" in str(ei.value)
    with pytest.raises(pt.PtError):
        pt.pt_energy_noalloc(0, "fp32", 4, 1, d_J.data_ptr(), d_H.data_ptr())
    with pytest.raises(pt.PtError):
        pt.pt_energy_noalloc(d_J.data_ptr(), "fp32", 1, 1, d_J.data_ptr(), d_H.data_ptr())
    pt.pt_energy_noalloc(d_J.data_ptr(), "fp32", 4, 0, d_J.data_ptr(), d_H.data_ptr())
