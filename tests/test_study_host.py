"""Host-side reductions of the study module: the integrated autocorrelation
time against the closed form of an AR(1) process, and the paper's ladder."""
import numpy as np
import pytest

from paper_1006_4247_gb300 import study


@pytest.mark.parametrize("rho", [0.0, 0.5, 0.8, 0.95])
def test_tau_int_of_ar1_process(rho):
    # x_t = rho x_{t-1} + e_t: rho(t) = rho^t, tau_int = (1 + rho) / (2 (1 - rho))
    rng = np.random.default_rng(1)
    n = 400_000
    e = rng.standard_normal(n)
    x = np.empty(n)
    x[0] = e[0]
    for t in range(1, n):
        x[t] = rho * x[t - 1] + e[t]
    want = (1 + rho) / (2 * (1 - rho))
    # windowing truncates the tail: bias ~ rho^W, statistical error ~ sqrt(2 (2W + 1) / n) tau
    assert study.tau_int(x) == pytest.approx(want, rel=0.06)


def test_tau_int_short_or_constant_series():
    assert np.isnan(study.tau_int(np.arange(4.0)))
    assert np.isnan(study.tau_int(np.ones(100)))


def test_paper_ladder():
    b = study.paper_ladder(15)
    assert b[0] == pytest.approx(1 / 0.19) and b[-1] == pytest.approx(1 / 0.12)
    # equal temperature ratios (section IV)
    T = 1 / b
    np.testing.assert_allclose(T[1:] / T[:-1], (0.12 / 0.19) ** (1 / 14))
