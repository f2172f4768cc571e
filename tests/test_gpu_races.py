"""Race checks of the checkerboard half sweeps with a poisoned colour.

A half sweep of one colour may read only the other colour's spins (and, for
overrelaxation, the old spin of the site itself): that is what makes the
checkerboard update of Section III.C parallel.  A kernel that read a spin of
the colour it is writing (a wrong halo index, a missing barrier between the
two colours, a slab that another CTA is still writing) would make its output
depend on values that the update must not see.  These tests change exactly
those values and check that nothing else moves:

* heat bath: the new spin does not depend on the old one (Eq. 5 draws it
  from the field alone), so after one full sweep (colour 0, then colour 1)
  the state is a function of the colour-1 input, the couplings, the betas and
  the random numbers only.  Replacing every colour-0 spin by another unit
  vector must give a bit-identical state and bit-identical energies;
* overrelaxation: the reflection of Eq. 7 at site x reads s_x and the six
  neighbours of the other colour, so after one sweep a change of a sparse set
  of colour-0 spins may only show at those sites (colour 0) and at their
  neighbours (colour 1).

Each case runs on the update path the engine picks for it (single-CTA
resident, clusters of 1024- or 512-thread CTAs, streaming with vector loads,
streaming with bulk copies), checked through the launch counts."""
import os

import numpy as np
import pytest

from gpu_util import get_state, make_engine, set_random_state, site_colour
from paper_1006_4247_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1006_4247_gb300 import _build
    _build.build()


S, C, NT = 2, 2, 3

# (L, precision, policy, environment, which resident path must run: None = none)
CASES = [
    (8, "fp32", "auto", {}, "resident"),
    (16, "fp32", "auto", {}, "resident"),
    (24, "fp32", "auto", {}, "resident"),
    (32, "fp32", "auto", {}, "resident"),
    (16, "fp64", "auto", {}, "resident"),
    (32, "fp64", "auto", {}, "resident"),
    (12, "fp32", "streaming", {}, None),
    (16, "fp32", "streaming", {}, None),
    (32, "fp32", "streaming", {}, None),
    (20, "fp64", "streaming", {}, None),
    (32, "fp32", "streaming", {"PT_TMA": "1"}, None),
    (32, "fp32", "auto", {"PT_CL_NARROW": "1"}, "resident"),
    (24, "fp64", "auto", {"PT_CL_NARROW": "1"}, "resident"),
]
IDS = [f"L{c[0]}-{c[1]}-{c[2]}" + "".join("-" + k[3:].lower() for k in c[3]) for c in CASES]


def _engine(L, precision, policy, env):
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        eng, J, B = make_engine(L, S, NT, C, precision, seed=23)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    eng.set_policy(policy)
    return eng


def _set_state(eng, L, st):
    for s in range(S):
        for c in range(C):
            for b in range(NT):
                eng.set_spins(s, c, b, st[s, c, b])


def _run(eng, L, st, step, n_hb, n_or):
    _set_state(eng, L, st)
    eng.step = step
    eng.profile(True)
    eng.sweep(n_hb, n_or)
    _, n = eng.profile_read()
    eng.profile(False)
    return get_state(eng, S, C, NT), eng.energies(), n


def _check_path(n, resident):
    if resident:
        assert n["resident"] >= 1, n
    else:
        assert n["resident"] == 0, n


def _neighbours(L, x):
    i, j, k = x % L, (x // L) % L, x // (L * L)
    out = []
    for di, dj, dk in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
        out.append((i + di) % L + L * ((j + dj) % L) + L * L * ((k + dk) % L))
    return out


@pytest.mark.parametrize("L,precision,policy,env,resident", CASES, ids=IDS)
def test_heat_bath_sweep_ignores_poisoned_colour(L, precision, policy, env, resident):
    eng = _engine(L, precision, policy, env)
    st = set_random_state(eng, S, C, NT, L, seed=41)
    step = eng.step
    a, Ha, n = _run(eng, L, st, step, 1, 0)
    _check_path(n, resident)
    poisoned = st.copy()
    m = site_colour(L) == 0
    for s in range(S):
        for c in range(C):
            for b in range(NT):
                poisoned[s, c, b][m] = W.random_spins(L, 900 + 100 * s + 10 * c + b)[m]
    assert np.abs(poisoned - st).max() > 0.5
    p, Hp, _ = _run(eng, L, poisoned, step, 1, 0)
    assert (p == a).all()
    assert (Hp == Ha).all()
    eng.close()


@pytest.mark.parametrize("L,precision,policy,env,resident", CASES, ids=IDS)
def test_overrelaxation_sweep_moves_only_near_perturbed_sites(L, precision, policy, env, resident):
    eng = _engine(L, precision, policy, env)
    st = set_random_state(eng, S, C, NT, L, seed=43)
    step = eng.step
    a, _, n = _run(eng, L, st, step, 0, 1)
    _check_path(n, resident)
    rng = np.random.default_rng(L)
    c0 = np.nonzero(site_colour(L) == 0)[0]
    picked = rng.choice(c0, size=max(2, c0.size // 32), replace=False)
    allowed = np.zeros(L ** 3, bool)
    allowed[picked] = True
    for x in picked:
        allowed[_neighbours(L, x)] = True
    pert = st.copy()
    fresh = W.random_spins(L, 77)
    pert[:, :, :, picked] = fresh[picked]
    p, _, _ = _run(eng, L, pert, step, 0, 1)
    moved = np.abs(p - a).max(axis=-1) > 0  # [S, C, NT, sites]
    assert not moved[..., ~allowed].any()
    assert moved[..., picked].all()
    eng.close()
