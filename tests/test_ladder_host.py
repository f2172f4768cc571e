"""Host logic of the learned ladder (paper_1006_4247_gb300/ladder.py) and the
CPU-side checks of the pt_mlp_* entry points: closed forms of the features,
the epsilon bound, the equal-acceptance construction and the kappa fit."""
import ctypes as C
import math

import numpy as np
import pytest

from paper_1006_4247_gb300 import ladder as lad


def test_coupling_statistic_closed_forms():
    L = 4
    J = np.full((3, L ** 3), -0.7, np.float32)
    assert lad.coupling_statistic(L, J) == pytest.approx(1.0, rel=1e-12)
    # Gaussian couplings: E sqrt(chi^2_6) / sqrt(6) = sqrt(2) Gamma(7/2) / Gamma(3) / sqrt(6)
    want = math.sqrt(2) * math.gamma(3.5) / math.gamma(3.0) / math.sqrt(6)
    J = np.random.default_rng(0).standard_normal((3, 24 ** 3)).astype(np.float32)
    assert lad.coupling_statistic(24, J) == pytest.approx(want, abs=0.005)


def test_coupling_statistic_counts_both_bond_directions():
    L = 4
    J = np.zeros((3, L ** 3), np.float32)
    J[0, 0] = 1.0  # one bond between site 0 and site 1 (x direction)
    # two sites carry sqrt(1) = 1, the rest 0; rms J = sqrt(1 / (3 L^3))
    want = (2.0 / L ** 3) / (math.sqrt(6.0) * math.sqrt(1.0 / (3 * L ** 3)))
    assert lad.coupling_statistic(L, J) == pytest.approx(want, rel=1e-12)


def test_eps_bound_by_hand():
    L = 4
    J = np.full((3, L ** 3), 0.5, np.float32)
    J[2, 5] = -2.0  # sites 5 and 5 + 16 now carry 5 * 0.5 + 2 = 4.5
    assert lad.eps_bound(L, J) == pytest.approx(lad.EPS_SAFETY / 4.5)


def test_geometric_and_default_count():
    b = lad.geometric(2.0, 8.0, 24)
    assert b[0] == 2.0 and b[-1] == pytest.approx(8.0)
    np.testing.assert_allclose(b[1:] / b[:-1], 4.0 ** (1 / 23))
    # the paper's ladders, T in [0.12, 0.19]
    assert lad.default_n_temps(16, 1 / 0.19, 1 / 0.12) == 15
    assert lad.default_n_temps(24, 1 / 0.19, 1 / 0.12) == 27
    assert lad.default_n_temps(4, 2.0, 2.5) == 3


def test_eps_from_kappa_caps():
    b = lad.geometric(2.0, 8.0, 5)
    e = lad.eps_from_kappa(b, [0.5, 0.5, 10.0, 0.5], 0.3)
    d = math.log(4.0) / 4
    np.testing.assert_allclose(e, [0.5 * d, 0.5 * d, 0.3, 0.5 * d], rtol=1e-6)


def test_equal_acceptance_shape_constant_is_geometric():
    b = lad.geometric(2.0, 8.0, 12)
    f = lad.equal_acceptance_shape(b, np.full(11, 0.4), 16)
    np.testing.assert_allclose(f, 1 / 16, rtol=1e-12)


def test_equal_acceptance_shape_equalises_a_model_density():
    # rejection density lambda(l) per unit ln beta, a smooth model
    lam = lambda l: 2.0 + 6.0 * np.exp(-((l - 1.2) / 0.2) ** 2)
    lb0, lb1 = math.log(2.0), math.log(8.0)

    def sigma(a, b, n=2000):
        t = np.linspace(a, b, n)
        return np.trapezoid(lam(t), t)

    # acceptance of a fine geometric ladder under the Gaussian model
    fine = lad.geometric(2.0, 8.0, 200)
    lf = np.log(fine)
    from scipy.special import erfc
    acc = erfc(np.array([sigma(lf[i], lf[i + 1]) for i in range(199)]) / (2 * math.sqrt(2)))
    f = lad.equal_acceptance_shape(fine, acc, 32)
    b = lad.shape_ladder(2.0, 8.0, f, 17)
    lb = np.log(b)
    s = np.array([sigma(lb[i], lb[i + 1]) for i in range(16)])
    assert s.std() / s.mean() < 0.02
    # more replicas where the density is high: the spacing shrinks near l = 1.2
    gaps = np.diff(lb)
    mid = 0.5 * (lb[1:] + lb[:-1])
    assert gaps[np.argmin(np.abs(mid - 1.2))] < 0.6 * gaps.max()
    assert lb[0] == pytest.approx(lb0) and lb[-1] == pytest.approx(lb1)


def test_best_kappa_recovers_parabola_vertex():
    k = np.array(lad.KAPPA_GRID)
    verts = np.array([0.06, 0.09, 0.115, 0.16])
    A = 0.6 - 0.3 * (k[:, None] - verts[None]) ** 2
    best, amax = lad.best_kappa(k, A)
    np.testing.assert_allclose(best, verts, atol=1e-12)
    np.testing.assert_allclose(amax, A.max(0))
    # maximum at the edge of the grid stays at the edge
    best, _ = lad.best_kappa(k, -(k[:, None] - 3.0) ** 2)
    assert best[0] == k[-1]


def test_mlp_entry_points_reject_bad_arguments_on_host():
    from paper_1006_4247_gb300 import _build, pt
    _build.build()
    lib = pt.load_library()
    h = C.c_void_p()
    assert lib.pt_mlp_create(C.byref(h), 0, 1, None) == pt.PT_ERR_ARG
    assert lib.pt_mlp_create(C.byref(h), pt.MLP_MAX_KNOTS + 1, 1, None) == pt.PT_ERR_ARG
    assert "n_knots" in pt.pt_last_error()
    assert lib.pt_mlp_create(None, 4, 1, None) == pt.PT_ERR_ARG
    assert lib.pt_mlp_num_params(None) == 0
    assert lib.pt_mlp_destroy(None) == pt.PT_OK
    x = np.zeros(4, np.float32)
    z = np.zeros(8, np.float32)
    fp = C.POINTER(C.c_float)
    assert lib.pt_mlp_forward(None, 1, x.ctypes.data_as(fp), z.ctypes.data_as(fp)) == pt.PT_ERR_ARG
    assert lib.pt_mlp_set_params(None, None) == pt.PT_ERR_ARG
    assert lib.pt_mlp_train(None, 1, None, None, C.c_float(1.0), 1, C.c_float(1e-3), None) == pt.PT_ERR_ARG


def test_parameter_count_matches_oracle_layout():
    from oracle import mlp as om
    from paper_1006_4247_gb300 import pt
    for P in (1, 5, 16, 64):
        assert pt.mlp_num_params(P) == om.layout(P)["total"]
