"""Long-run statistical parity of the GPU engine with the FP64 oracle, and the
closed forms of the update cycle on the GPU.

Workload of the long runs: L = 4 periodic, Gaussian couplings (seed 1),
8 inverse temperatures linear in [2.5, 8.0], two copies, 1 heat-bath + 3
overrelaxation sweeps per cycle then one tempering update, 1000 cycles, the
first 200 discarded.  The GPU runs 96 independent chain pairs of the same
coupling set (one per sample slot, each with its own Philox key); the oracle
side is 96 independent oracle runs stored in tests/golden/stats_L4_R8.json by
tests/golden/make_stats_L4.py.  Errors come from the spread over independent
runs.  Rule (23 observables at once): at least 90% within 2 sigma and all
within 4.5 sigma of the combined error, for <H>(beta), <chi>(beta) and the
acceptance of every pair.
"""
import json
import os

import numpy as np
import pytest

import oracle as orc
from paper_1006_4247_gb300 import pt
from paper_1006_4247_gb300 import workloads as W

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
L, NT = 4, 8
BETAS = W.linear_betas(NT, 2.5, 8.0)
CYCLES, BURN = 1000, 200
MODES = {"plain": (0, 0.0), "decimation": (1, 0.0), "coolheat": (2, 0.05)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1006_4247_gb300 import _build
    _build.build()


def _gpu_run(mode, precision, S=96, seed=1234, eps=None):
    J = W.couplings(L, 1)
    eng = pt.Engine(L, np.stack([J] * S), np.stack([BETAS] * S), n_copies=2, precision=precision, seed=seed)
    e = MODES[mode][1] if eps is None else eps
    eng.set_params(eps=np.full(S * (NT - 1), e, np.float32))
    H = np.zeros((CYCLES, S, 2, NT))
    chi = np.zeros((CYCLES, S, NT))
    for c in range(CYCLES):
        eng.sweep(1, 3)
        eng.exchange(mode)
        h, q, x = eng.measure()
        H[c] = h.reshape(S, 2, NT)
        chi[c] = x.reshape(S, NT)
    prop, acc, rt, perm = eng.stats()
    eng.close()
    # per independent run: <H>(beta) over both copies, <chi>(beta), acceptance
    return (H[BURN:].mean(axis=(0, 2)), chi[BURN:].mean(axis=0),
            (acc / np.maximum(prop, 1)).mean(axis=1))


def _oracle_stats(mode):
    with open(os.path.join(HERE, "golden", "stats_L4_R8.json")) as fh:
        d = json.load(fh)
    assert d["L"] == L and d["NT"] == NT and np.allclose(d["betas"], BETAS)
    m = d["modes"][mode]
    return np.array(m["H"]), np.array(m["chi"]), np.array(m["acc"])


def _z(a, b):
    ma, ea = a.mean(0), a.std(0, ddof=1) / np.sqrt(a.shape[0])
    mb, eb = b.mean(0), b.std(0, ddof=1) / np.sqrt(b.shape[0])
    return np.abs(ma - mb) / np.sqrt(ea ** 2 + eb ** 2), ma, mb, np.sqrt(ea ** 2 + eb ** 2)


@pytest.mark.parametrize("mode", ["plain", "decimation", "coolheat"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_long_run_observables_match_oracle(mode, precision):
    seed = 1234 if precision == "fp64" else 4321
    g = _gpu_run(mode, precision, seed=seed)
    o = _oracle_stats(mode)
    parts = [_z(a, b) for a, b in zip(g, o)]
    z = np.concatenate([p[0] for p in parts])
    msg = "\n".join(f"{n}: gpu {np.round(p[1], 4)} oracle {np.round(p[2], 4)} err {np.round(p[3], 4)} z {np.round(p[0], 2)}"
                    for n, p in zip(("H", "chi", "acc"), parts))
    assert np.isfinite(z).all(), msg
    assert (z < 2.0).mean() >= 0.9, msg
    assert z.max() < 4.5, msg


def test_modified_exchange_doubles_acceptance_on_gpu():
    """Trend of section IV.A on the GPU: decimation and cooling/heating are
    accepted more often than the standard swap at the same ladder."""
    acc = {m: _gpu_run(m, "fp32", S=16, eps=0.01)[2].mean() for m in ("plain", "decimation", "coolheat")}
    assert acc["decimation"] > 1.3 * acc["plain"]
    assert acc["coolheat"] > acc["plain"]


def test_beta_zero_closed_forms_gpu():
    """beta = 0: every heat-bath sweep draws uniform spins, so <H> = 0,
    Var H = sum_b J_b^2 / 3 and <chi> = 1 (replica 0, no exchanges)."""
    S = 64
    Js = np.stack([W.couplings(L, 61)] * S)
    eng = pt.Engine(L, Js, np.stack([np.array([0.0, 0.5])] * S), n_copies=2, precision="fp32", seed=3)
    Hs, chis = [], []
    for _ in range(200):
        eng.sweep(1, 0)
        h, q, x = eng.measure()
        Hs.append(h.reshape(S, 2, 2)[:, :, 0].ravel())
        chis.append(x.reshape(S, 2)[:, 0])
    eng.close()
    H = np.concatenate(Hs)
    chi = np.concatenate(chis)
    var = (Js[0].astype(np.float64) ** 2).sum() / 3
    assert abs(H.mean()) < 5 * np.sqrt(var / H.size)
    assert abs(H.var() - var) < 5 * np.sqrt(2.0 / H.size) * var
    assert abs(chi.mean() - 1.0) < 5 * chi.std() / np.sqrt(chi.size)


def test_high_temperature_series_gpu():
    """<H> at beta = 0.1, 0.2, 0.3 against the high-temperature series of
    ln Z (single-bond Langevin terms plus closed loops through six bonds,
    L = 4), allowing for the omitted graphs the size of the six-bond order."""
    from test_oracle_thermo import _highT_energy, _highT_remainder
    S = 64
    J = W.couplings(L, 74)
    betas = np.array([0.1, 0.2, 0.3])
    eng = pt.Engine(L, np.stack([J] * S), np.stack([betas] * S), n_copies=2, precision="fp64", seed=8)
    Hs = []
    for c in range(600):
        eng.sweep(1, 1)
        eng.exchange("plain")
        if c >= 100:
            Hs.append(eng.energies().mean(axis=1))  # [S, 3]
    eng.close()
    per_chain = np.stack(Hs).mean(0)  # [S, 3]
    m, e = per_chain.mean(0), per_chain.std(0, ddof=1) / np.sqrt(S)
    for b, beta in enumerate(betas):
        ref = _highT_energy(L, J.astype(np.float64), beta)
        rem = _highT_remainder(L, J.astype(np.float64), beta)
        assert abs(m[b] - ref) < 4.5 * e[b] + rem, (beta, m[b], ref, e[b], rem)
