"""Pins of the FP64 oracle of the ladder network (oracle/mlp.py) against what
fixes it independently of its own code: a network computed by hand, central
finite differences of the loss, the closed-form first Adam step, bfloat16 bit
patterns made by hand and torch's conversion, and closed forms of the
decoding (geometric ladder, constant kappa)."""
import numpy as np
import pytest

from oracle import mlp as om

P = 5


def _random_params(rng, P, scale=0.5):
    n = om.layout(P)["total"]
    return rng.standard_normal(n) * scale


def _rows(rng, B, P):
    x = np.stack([np.log(rng.choice([4, 8, 16], B)), rng.uniform(1.5, 3, B), rng.uniform(5, 9, B),
                  rng.uniform(0.9, 1.0, B)], axis=1)
    f = rng.dirichlet(np.ones(P), B)
    e = rng.uniform(0.05, 0.95, (B, P))
    lam = rng.uniform(1.0, 4.0, (B, 1))
    return x, np.concatenate([f, e, lam], axis=1)


def test_forward_hand_network():
    W1 = np.zeros((64, 4)); W1[0, 0] = 1.0; W1[1, 1] = -1.0
    b1 = np.zeros(64); b1[2] = 0.5
    W2 = np.zeros((64, 64)); W2[0, 0] = 2.0; W2[1, 1] = 3.0; W2[2, 2] = -1.0
    b2 = np.zeros(64)
    W3 = np.zeros((3, 64)); W3[0, 0] = 1.0; W3[0, 1] = 1.0; W3[1, 2] = 1.0; W3[2, 1] = -0.5
    b3 = np.array([0.25, -0.5, 1.0])
    p = om.pack(W1, b1, W2, b2, W3, b3)
    z, (h1, h2) = om.forward(p, np.array([[1.5, -2.0, 0.0, 0.0]]), 1)
    # h1 = (1.5, 2, 0.5, 0...), h2 = (3, 6, relu(-0.5) = 0, ...)
    assert h1[0, :3].tolist() == [1.5, 2.0, 0.5]
    assert h2[0, :3].tolist() == [3.0, 6.0, 0.0]
    assert z[0].tolist() == [9.25, -0.5, -2.0]


def test_loss_single_knot_by_hand():
    # P = 1: the only shape fraction is 1, so the loss is
    # (1 - t0)^2 + w (sigmoid(z1) - t1)^2 + (z2 - t2)^2
    p = np.zeros(om.layout(1)["total"])
    lay = om.layout(1)
    p[lay["b3"][0]:lay["b3"][0] + 3] = [0.3, 0.0, 1.5]  # z = (0.3, 0, 1.5) for every input
    x = np.zeros((2, 4))
    t = np.array([[0.6, 0.2, 1.0], [1.0, 0.5, 1.5]])
    want = np.mean([(1 - 0.6) ** 2 + 2.0 * (0.5 - 0.2) ** 2 + 0.25, 0.0 + 2.0 * 0.0 + 0.0])
    assert om.loss(p, x, t, 1, 2.0) == pytest.approx(want, rel=1e-15)


def test_loss_and_gradient_vanish_at_own_outputs():
    rng = np.random.default_rng(1)
    p = _random_params(rng, P)
    x, _ = _rows(rng, 6, P)
    z, _ = om.forward(p, x, P)
    t = np.concatenate([om.shape_fractions(z, P), om.sigmoid(z[:, P:2 * P]), z[:, 2 * P:]], axis=1)
    L, g = om.loss_grad(p, x, t, P, 0.7)
    assert L == pytest.approx(0.0, abs=1e-28)
    assert np.abs(g).max() < 1e-14


@pytest.mark.parametrize("w_kappa", [0.0, 1.0, 3.0])
def test_gradient_matches_central_differences(w_kappa):
    rng = np.random.default_rng(7)
    p = _random_params(rng, P)
    x, t = _rows(rng, 7, P)
    L, g = om.loss_grad(p, x, t, P, w_kappa)
    assert L == pytest.approx(om.loss(p, x, t, P, w_kappa), rel=1e-14)
    h = 1e-6
    fd = np.empty_like(p)
    for i in range(p.size):
        a, b = p.copy(), p.copy()
        a[i] += h
        b[i] -= h
        fd[i] = (om.loss(a, x, t, P, w_kappa) - om.loss(b, x, t, P, w_kappa)) / (2 * h)
    assert np.abs(fd - g).max() <= 1e-7 * np.abs(g).max() + 1e-10
    # every parameter block receives gradient (no block dropped)
    lay = om.layout(P)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        a, n = lay[k]
        if w_kappa == 0.0 and k == "b3":
            assert np.abs(g[a:a + P]).max() > 0 and g[a + 2 * P] != 0  # no kappa part
            assert np.abs(g[a + P:a + 2 * P]).max() == 0
        else:
            assert np.abs(g[a:a + n]).max() > 0, k


def test_adam_first_steps_closed_form():
    rng = np.random.default_rng(3)
    p0 = rng.standard_normal(50)
    g = rng.standard_normal(50)
    m = v = np.zeros(50)
    p1, m, v = om.adam_step(p0, m, v, g, 1, 0.01)
    # bias-corrected moments equal g and g^2 after one step
    np.testing.assert_allclose(p1, p0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    # with a constant gradient the corrected moments stay g, g^2
    p2, m, v = om.adam_step(p1, m, v, g, 2, 0.01)
    np.testing.assert_allclose(p2, p1 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-14)


def test_bf16_rounding_bit_patterns():
    bits = np.array([0x3F800000, 0x3F808000, 0x3F818000, 0x3F808001, 0x3F807FFF, 0xBFC00000, 0x3F7FFFFF,
                     0x00000000, 0x80000000], np.uint32)
    want = [0x3F80, 0x3F80, 0x3F82, 0x3F81, 0x3F80, 0xBFC0, 0x3F80, 0x0000, 0x8000]
    assert om.bf16_bits(bits.view(np.float32)).tolist() == want
    assert om.bf16_value(np.array([0x3F80, 0xC040], np.uint16)).tolist() == [1.0, -3.0]


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    a = np.random.default_rng(5).standard_normal(20000).astype(np.float32) * 10.0 ** np.random.default_rng(
        6).integers(-8, 8, 20000)
    a = a.astype(np.float32)
    t = torch.from_numpy(a).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert (om.bf16_bits(a) == t).all()


@pytest.mark.parametrize("NT", [2, 7, 17, 48])
def test_decode_equal_shape_is_geometric(NT):
    P = 16
    z = np.concatenate([np.full(P, 0.37), np.full(P, -0.4), [0.0]])
    b, e = om.decode(z, P, 2.0, 8.0, NT, 2.0)
    want = 2.0 * 4.0 ** (np.arange(NT) / (NT - 1))
    np.testing.assert_allclose(b, want, rtol=1e-14)
    assert b[0] == 2.0 and b[-1] == 8.0
    # constant kappa: eps_i = kappa_max sigmoid(c) ln(beta_{i+1}/beta_i)
    np.testing.assert_allclose(e, 2.0 / (1 + np.exp(0.4)) * np.log(4.0) / (NT - 1), rtol=1e-13)


def test_decode_random_outputs():
    rng = np.random.default_rng(11)
    P = 16
    for _ in range(20):
        z = rng.standard_normal(2 * P + 1) * 2
        NT = int(rng.integers(2, 60))
        b, e = om.decode(z, P, 1.7, 6.3, NT, 1.5)
        assert b[0] == 1.7 and b[-1] == 6.3
        assert (np.diff(b) > 0).all()
        assert (e > 0).all() and (e <= 1.5 * np.diff(np.log(b)) + 1e-15).all()
    # NT - 1 = P: the replicas sit on the knots, ln beta_k = ln b0 + span * sum_{j<k} f_j
    z = rng.standard_normal(2 * P + 1)
    b, _ = om.decode(z, P, 2.0, 8.0, P + 1, 1.0)
    f = np.log1p(np.exp(z[:P])) + np.float64(np.float32(0.01))
    f /= f.sum()
    want = np.log(2.0) + np.log(4.0) * np.concatenate([[0.0], np.cumsum(f)])
    np.testing.assert_allclose(np.log(b), want, rtol=0, atol=1e-14)


def test_replica_count_closed_form():
    P = 4
    z = np.zeros(2 * P + 1)
    z[2 * P] = np.log(10.5)
    # Lambda = 10.5: sigma 2 -> 1 + ceil(5.25) = 7; sigma 3 -> 1 + ceil(3.5) = 5; clamps
    assert om.replica_count(z, P, 2.0, 100) == 7
    assert om.replica_count(z, P, 3.0, 100) == 5
    assert om.replica_count(z, P, 0.1, 50) == 50
    z[2 * P] = -30.0
    assert om.replica_count(z, P, 1.0, 50) == 2
