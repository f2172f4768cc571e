"""Pins of the oracle's replica exchanges: the standard swap (Eq. 1), the
decimation swap (section III.A, Eq. aswap, appendix A) and the cooling/heating
swap (section III.B), plus the round-trip bookkeeping of section IV.B."""
import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss

from paper_1006_4247_gb300 import workloads as W


# --------------------------------------------------------------------------
# standard swap
# --------------------------------------------------------------------------
def _chain(orc, L, betas, seed=5, copy=0, sample=0, spins=None):
    NT = len(betas)
    J = W.couplings(L, 40).astype(np.float64)
    if spins is None:
        spins = W.random_spins(L, seed, NT)
    return orc.Chain(L, J, betas, spins, copy=copy, sample=sample, seed=seed)


def test_plain_swap_rule_exact(orc):
    """Accept iff Delta >= 0 or u < exp(Delta), Delta = (b_{i+1}-b_i)(H_{i+1}-H_i),
    pairs in increasing beta, each seeing the previous result."""
    L = 2
    betas = np.array([0.5, 1.0, 1.7, 2.0])
    for step in range(200):
        ch = _chain(orc, L, betas, seed=step)
        H = ch.H.copy()
        lab = ch.label.copy()
        ch.exchange(0, step)
        # replay by hand
        for i in range(3):
            d = (betas[i + 1] - betas[i]) * (H[i + 1] - H[i])
            w = orc.rng_words(ch.seed, 0, i, 0, step, 1)
            u = ((int(w[0]) >> 5) * 67108864.0 + (int(w[1]) >> 6)) * 2.0 ** -53
            if d >= 0 or u < np.exp(d):
                H[[i, i + 1]] = H[[i + 1, i]]
                lab[[i, i + 1]] = lab[[i + 1, i]]
        assert (ch.label == lab).all()
        assert np.allclose(ch.H, H)


def test_plain_swap_acceptance_frequency(orc):
    """With fixed energies the acceptance frequency is min(1, e^Delta)."""
    L = 2
    betas = np.array([1.0, 1.25])
    ch = _chain(orc, L, betas)
    J = ch.J
    s = ch.spins.copy()
    H = [orc.energy(L, J, s[b]) for b in range(2)]
    # order the two configs so that Delta < 0
    if (betas[1] - betas[0]) * (H[1] - H[0]) > 0:
        s = s[::-1].copy()
    n = 20000
    acc = 0
    for step in range(n):
        c = orc.Chain(L, J, betas, s, seed=3)
        c.exchange(0, step)
        acc += int(c.acc[0])
    Hs = [orc.energy(L, J, s[b]) for b in range(2)]
    p = min(1.0, np.exp((betas[1] - betas[0]) * (Hs[1] - Hs[0])))
    assert abs(acc / n - p) < 5 * np.sqrt(p * (1 - p) / n)


def test_roundtrip_counting(orc):
    """A round trip is index 0 -> index NT-1 -> index 0 of one configuration."""
    NT = 3
    label = np.array([0, 1, 2], np.int32)
    rs = np.zeros(NT, np.int32)
    rs[0] = 1
    cnt = np.zeros(1, np.int64)
    seq = [[1, 0, 2], [1, 2, 0], [0, 2, 1], [2, 0, 1], [0, 2, 1], [0, 1, 2], [2, 1, 0]]
    counts = []
    for lab in seq:
        label[:] = lab
        orc.roundtrip_update(label, rs, cnt)
        counts.append(int(cnt[0]))
    # label 0: top (start) -> bottom (state 1) -> top (state 2): trip 1
    # label 2: top (state 3) -> bottom (state 5) -> top (state 6): trip 2
    assert counts == [0, 0, 1, 1, 1, 1, 2]
    label[:] = [2, 1, 0]
    orc.roundtrip_update(label, rs, cnt)  # nothing new
    label[:] = [0, 1, 2]
    orc.roundtrip_update(label, rs, cnt)  # label 0: top (2) -> bottom (6) -> top: trip 3
    assert cnt[0] == 3


# --------------------------------------------------------------------------
# decimation
# --------------------------------------------------------------------------
def _ln_I_over_4pi(R, n=400):
    """ln( (1/2) int_{-1}^{1} e^{R c} dc ) by Gauss-Legendre, scaled for large R."""
    x, w = leggauss(n)
    return R + np.log(0.5 * (w * np.exp(R * (x - 1))).sum())


@pytest.mark.parametrize("R", [0.0, 1e-8, 1e-3, 0.3, 0.5, 0.9, 1.0, 3.0, 17.4, 17.6, 40.0, 300.0])
def test_ln_sinhc_vs_quadrature(orc, R):
    """ln I(beta S)/(4 pi) = ln(sinh R / R) (Eq. HI)."""
    assert abs(orc.ln_sinhc(R) - _ln_I_over_4pi(R)) < 1e-12 * max(1.0, R)


def test_decimation_ratio_vs_quadrature(orc):
    """Eq. aswap: ln A = sum over decimated x of ln I(b2 S1) - ln I(b1 S1)
    + ln I(b1 S2) - ln I(b2 S2), with S from the kept colour."""
    L = 4
    J = W.couplings(L, 8).astype(np.float64)
    s1, s2 = W.random_spins(L, 1), W.random_spins(L, 2)
    b1, b2 = 2.1, 2.6
    x = np.arange(L ** 3)
    col = ((x % L) + (x // L) % L + x // (L * L)) % 2
    for d in (0, 1):
        ref = 0.0
        for xi in x[col == d]:
            a = np.linalg.norm(orc.local_field(L, J, s1, xi))
            b = np.linalg.norm(orc.local_field(L, J, s2, xi))
            ref += (_ln_I_over_4pi(b2 * a) - _ln_I_over_4pi(b1 * a)
                    + _ln_I_over_4pi(b1 * b) - _ln_I_over_4pi(b2 * b))
        got = orc.decimation_lnA(L, J, s1, s2, d, b1, b2)
        assert abs(got - ref) < 1e-9 * max(1, abs(ref))
        assert orc.decimation_lnA(L, J, s1, s2, d, b1, b1) == 0.0


def test_decimation_kept_colour_swapped_and_reinserted(orc):
    """On acceptance the kept colour of the two configs is exchanged and the
    decimated colour is redrawn; on rejection nothing changes."""
    L = 4
    betas = np.array([2.0, 2.05])
    x = np.arange(L ** 3)
    col = ((x % L) + (x // L) % L + x // (L * L)) % 2
    seen = {True: 0, False: 0}
    for step in range(40):
        ch = _chain(orc, L, betas, seed=100 + step)
        before = ch.spins.copy()
        ch.exchange(1, step)
        w = orc.rng_words(ch.seed, 0, 0, 0, step, 3)
        d = int(w[0]) & 1
        accepted = bool(ch.acc[0])
        seen[accepted] += 1
        if accepted:
            assert (ch.spins[0][col != d] == before[1][col != d]).all()
            assert (ch.spins[1][col != d] == before[0][col != d]).all()
            assert (ch.label == [1, 0]).all()
            for b in range(2):
                assert abs(ch.H[b] - orc.energy(L, ch.J, ch.spins[b])) < 1e-12
        else:
            assert (ch.spins == before).all()
    assert seen[True] > 0 and seen[False] > 0


# --------------------------------------------------------------------------
# cooling / heating
# --------------------------------------------------------------------------
def _unit(v):
    return v / np.linalg.norm(v)


def test_cool_heat_site_inverse_and_angle(orc, rng):
    """The cooling step lowers the angle to S by alpha = eps |p|; heating
    undoes it (Newton on theta - e sin theta = theta')."""
    for _ in range(300):
        S = rng.standard_normal(3) * rng.uniform(0.1, 6)
        eps = rng.uniform(0.0, 0.9) / np.linalg.norm(S)
        s = _unit(rng.standard_normal(3))
        c, _ = orc.cool_site(eps, S, s)
        th = np.arccos(np.clip(_unit(S) @ s, -1, 1))
        thp = np.arccos(np.clip(_unit(S) @ c, -1, 1))
        alpha = eps * np.linalg.norm(S - (S @ s) * s)
        assert abs((th - thp) - alpha) < 1e-7
        # coplanar with s and S
        assert abs(np.linalg.det(np.stack([s, S, c]))) < 1e-10 * np.linalg.norm(S)
        back, _ = orc.heat_site(eps, S, c)
        assert np.allclose(back, s, atol=1e-12)


def test_cool_site_jacobian_vs_finite_difference(orc, rng):
    """det J_f = d cos(theta') / d cos(theta) = |1 - eps S.s|
    (cos alpha - cot theta sin alpha)."""
    for _ in range(100):
        S = rng.standard_normal(3) * rng.uniform(0.1, 6)
        nS = np.linalg.norm(S)
        eps = rng.uniform(0.0, 0.9) / nS
        n = S / nS
        e1 = _unit(np.cross(n, rng.standard_normal(3)))
        th = rng.uniform(0.05, np.pi - 0.05)
        h = 1e-6

        def cos_after(t):
            s = np.cos(t) * n + np.sin(t) * e1
            c, _ = orc.cool_site(eps, S, s)
            return c @ n

        s0 = np.cos(th) * n + np.sin(th) * e1
        _, lj = orc.cool_site(eps, S, s0)
        num = (cos_after(th + h) - cos_after(th - h)) / (np.cos(th + h) - np.cos(th - h))
        assert abs(np.exp(lj) - num) < 1e-6 * num


def test_kepler_newton_converges(orc):
    for e in list(np.linspace(0, 0.9, 10)) + [0.97, 0.99, 0.999]:
        for thp in np.linspace(0, np.pi, 41):
            th = orc.kepler_solve(e, thp)
            assert abs(th - e * np.sin(th) - thp) < 1e-13


def _sphere_coords(v):
    return np.stack([v[:, 2], np.arctan2(v[:, 1], v[:, 0])], 1)


def _from_coords(c):
    z, ph = c[:, 0], c[:, 1]
    r = np.sqrt(1 - z ** 2)
    return np.stack([r * np.cos(ph), r * np.sin(ph), z], 1)


def test_cool_sweep_jacobian_vs_numerical_determinant(orc):
    """ln det J_C of the whole cooling sweep (black then white) equals
    ln |det| of the numerically differentiated 2N-dimensional map in the
    area-preserving coordinates (z, phi) at L = 2."""
    L = 2
    N = L ** 3
    J = W.couplings(L, 31).astype(np.float64)
    rng = np.random.default_rng(5)
    for trial in range(3):
        s = W.random_spins(L, 50 + trial)
        s[:, 2] = np.clip(s[:, 2], -0.9, 0.9)
        s = s / np.linalg.norm(s, axis=1, keepdims=True)
        eps = 0.08
        _, lnJ = orc.cool_sweep(L, J, s, eps)
        c0 = _sphere_coords(s).ravel()
        h = 1e-6
        M = np.zeros((2 * N, 2 * N))
        for k in range(2 * N):
            cp, cm = c0.copy(), c0.copy()
            cp[k] += h
            cm[k] -= h
            fp, _ = orc.cool_sweep(L, J, _from_coords(cp.reshape(N, 2)), eps)
            fm, _ = orc.cool_sweep(L, J, _from_coords(cm.reshape(N, 2)), eps)
            dp = _sphere_coords(fp).ravel() - _sphere_coords(fm).ravel()
            dp[1::2] = (dp[1::2] + np.pi) % (2 * np.pi) - np.pi
            M[:, k] = dp / (2 * h)
        sign, logdet = np.linalg.slogdet(M)
        assert abs(logdet - lnJ) < 1e-5, (logdet, lnJ)


def test_cool_heat_sweep_inverse_and_jacobian_consistency(orc):
    L = 4
    J = W.couplings(L, 9).astype(np.float64)
    s = W.random_spins(L, 3)
    for eps in (0.0, 0.01, 0.05):
        c, lj_c = orc.cool_sweep(L, J, s, eps)
        back, lj_h = orc.heat_sweep(L, J, c, eps)
        assert np.abs(back - s).max() < 1e-12
        # heat_sweep returns ln det J_C at its result, which is s
        assert abs(lj_c - lj_h) < 1e-10
        if eps == 0.0:
            assert lj_c == 0.0 and np.abs(c - s).max() < 1e-15
        else:
            # cooling lowers the energy
            assert orc.energy(L, J, c) < orc.energy(L, J, s)


def test_coolheat_eps0_is_plain_swap(orc):
    L = 4
    J = W.couplings(L, 9).astype(np.float64)
    s1, s2 = W.random_spins(L, 3), W.random_spins(L, 4)
    H1, H2 = orc.energy(L, J, s1), orc.energy(L, J, s2)
    lnA, t1, t2, Hc, Hh = orc.coolheat_lnA(L, J, s1, s2, H1, H2, 1.5, 1.9, 0.0)
    assert abs(lnA - (1.9 - 1.5) * (H2 - H1)) < 1e-12
    betas = np.array([1.5, 1.9])
    for step in range(30):
        a = _chain(orc, L, betas, seed=step)
        b = _chain(orc, L, betas, seed=step)
        a.exchange(0, step)
        b.exchange(2, step, eps=0.0)
        assert (a.label == b.label).all() and (a.acc == b.acc).all()
