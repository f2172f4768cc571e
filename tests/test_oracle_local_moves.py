"""Pins of the oracle's single-site moves (section III.C of Hasenbusch &
Schaefer): heat bath by inversion of the conditional distribution of
cos(theta) ~ exp(R cos theta) on [-1, 1], and overrelaxation by reflection."""
import numpy as np
import pytest
from scipy import stats


def _cdf(R, c):
    """P(cos theta <= c) for density proportional to exp(R c) on [-1, 1]."""
    if R == 0:
        return (c + 1) / 2
    return (np.expm1(-R * (1 - c)) - np.expm1(-2 * R)) / (-np.expm1(-2 * R))


@pytest.mark.parametrize("R", [0.0, 1e-9, 1e-4, 0.01, 0.5, 1.0, 3.0, 20.0, 80.0, 150.0])
def test_hb_inverts_the_cdf(orc, R):
    """The new cos(theta) = 1 - t solves F(c) = r exactly (r = 1 - q)."""
    for m in [0, 1, 2, 1000, 2 ** 23, 2 ** 24 - 2, 2 ** 24 - 1]:
        q = (2 ** 24 - 1 - m) * 2.0 ** -24
        t = orc.hb_t(R, q)
        assert 0.0 <= t <= 2.0
        r = 1.0 - q
        assert abs(_cdf(R, 1.0 - t) - r) <= 1e-12 * max(1.0, R), (R, m)


@pytest.mark.parametrize("R", [0.3, 1.0, 5.0, 20.0])
def test_hb_matches_printed_formula(orc, R):
    """Section III.C: s_p = ln(z + (1/z - z) r) / R, z = exp(-R)."""
    z = np.exp(-R)
    for m in [0, 7, 12345, 2 ** 22, 2 ** 24 - 1]:
        r = (m + 1) * 2.0 ** -24
        sp = np.log(z + (1 / z - z) * r) / R
        t = orc.hb_t(R, 1.0 - r)
        assert abs((1.0 - t) - sp) < 1e-12


def _draw(orc, beta, S, n, seed):
    rng = np.random.default_rng(seed)
    w = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64)
    return np.array([orc.hb_update(beta, S, int(a), int(b)) for a, b in w])


@pytest.mark.parametrize("R", [0.0, 0.7, 2.0, 10.0])
def test_hb_distribution(orc, R):
    """Mean of cos(theta) is the Langevin function coth R - 1/R; KS test of the
    full distribution; the azimuth about S is uniform; |s| = 1."""
    n = 6000
    S = np.array([0.3, -1.2, 0.8])
    nS = np.linalg.norm(S)
    beta = R / nS
    s = _draw(orc, beta, S, n, seed=int(R * 10) + 1)
    assert np.allclose(np.linalg.norm(s, axis=1), 1.0, atol=1e-14)
    c = s @ (S / nS)
    mean = 0.0 if R == 0 else 1 / np.tanh(R) - 1 / R
    assert abs(c.mean() - mean) < 5 * c.std() / np.sqrt(n)
    ks = stats.kstest(c, lambda x: np.array([_cdf(R, v) for v in np.atleast_1d(x)]))
    assert ks.pvalue > 1e-4
    # azimuth in a fixed frame around n
    nvec = S / nS
    a = np.cross(nvec, [1.0, 0.0, 0.0]); a /= np.linalg.norm(a)
    b = np.cross(nvec, a)
    perp = s - np.outer(c, nvec)
    phi = np.arctan2(perp @ b, perp @ a)
    ks2 = stats.kstest((phi + np.pi) / (2 * np.pi), "uniform")
    assert ks2.pvalue > 1e-4


def test_hb_zero_field_is_uniform(orc):
    """S = 0: uniform on the sphere (Archimedes: z uniform in [-1, 1])."""
    s = _draw(orc, 1.0, np.zeros(3), 5000, seed=9)
    for a in range(3):
        assert stats.kstest((s[:, a] + 1) / 2, "uniform").pvalue > 1e-4


@pytest.mark.parametrize("n", [[0, 0, 1], [0, 0, -1], [1, 0, 0], [0.6, 0.8, 0.0],
                               [0.6, 0.8, -0.0], [1e-9, 0, -1 + 1e-18], [0.36, 0.48, 0.8]])
def test_onb_orthonormal(orc, n):
    n = np.array(n, float)
    n /= np.linalg.norm(n)
    e1, e2 = orc.onb(n)
    M = np.stack([e1, e2, n])
    assert np.allclose(M @ M.T, np.eye(3), atol=1e-12)
    assert np.linalg.det(M) > 0


def test_or_reflection(orc, rng):
    """s' = 2 (s.S)/S^2 S - s: involution, keeps s.S (so the local energy),
    |s'| = 1, and s + s' is parallel to S.  S = 0 leaves s unchanged."""
    for _ in range(200):
        S = rng.standard_normal(3) * rng.uniform(0.01, 5)
        s = rng.standard_normal(3); s /= np.linalg.norm(s)
        s1 = orc.or_update(S, s)
        assert abs(np.linalg.norm(s1) - 1) < 1e-14
        assert abs(s1 @ S - s @ S) < 1e-12 * np.linalg.norm(S)
        assert np.linalg.norm(np.cross(s + s1, S)) < 1e-12 * np.linalg.norm(S)
        assert np.allclose(orc.or_update(S, s1), s, atol=1e-14)
    s = np.array([0.0, 0.6, 0.8])
    assert (orc.or_update(np.zeros(3), s) == s).all()


def test_or_sweep_conserves_energy_hb_does_not(orc):
    from paper_1006_4247_gb300 import workloads as W
    L = 4
    J = W.couplings(L, 5).astype(np.float64)
    s = W.random_spins(L, 6)
    H0 = orc.energy(L, J, s)
    t = orc.or_halfsweep(L, J, s, 0)
    t = orc.or_halfsweep(L, J, t, 1)
    assert abs(orc.energy(L, J, t) - H0) < 1e-12 * abs(H0)
    assert np.abs(t - s).max() > 1e-3
    u = orc.hb_halfsweep(L, J, s, 0, 2.0, 1, 0, 0, 0)
    assert abs(orc.energy(L, J, u) - H0) > 1e-3


def test_halfsweep_touches_one_colour_only(orc):
    from paper_1006_4247_gb300 import workloads as W
    L = 4
    J = W.couplings(L, 5).astype(np.float64)
    s = W.random_spins(L, 6)
    x = np.arange(L ** 3)
    col = ((x % L) + (x // L) % L + x // (L * L)) % 2
    for c in (0, 1):
        t = orc.hb_halfsweep(L, J, s, c, 1.5, 3, 0, 0, 11)
        assert (t[col != c] == s[col != c]).all()
        assert (np.abs(t[col == c] - s[col == c]).max(axis=1) > 0).all()
