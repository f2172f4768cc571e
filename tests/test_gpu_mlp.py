"""Parity of the ladder network's kernels (pt_mlp_*) with the FP64 oracle
(oracle/mlp.py): the bfloat16 weight copy bit for bit, forward outputs,
loss and gradient through the bfloat16 weights, Adam steps, the decoding of
ladders and epsilons, and deterministic training on the device.

Batches of 100 rows span four backward chunks of 32 rows with a ragged tail."""
import numpy as np
import pytest

from oracle import mlp as om
from paper_1006_4247_gb300 import pt

pytestmark = pytest.mark.gpu

P = 16
B = 100


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1006_4247_gb300 import _build
    _build.build()


def _rows(rng, n, P=P):
    x = np.stack([np.log(rng.choice([4, 6, 8, 12, 16, 24, 32, 48], n)), rng.uniform(1.5, 3.0, n),
                  rng.uniform(5.0, 9.0, n), rng.uniform(0.93, 0.99, n)], axis=1).astype(np.float32)
    f = rng.dirichlet(np.full(P, 4.0), n)
    e = rng.uniform(0.1, 0.5, (n, P))
    lam = rng.uniform(2.0, 5.0, (n, 1))
    return x, np.concatenate([f, e, lam], axis=1).astype(np.float32)


def _net(seed=5, scale=0.3):
    net = pt.Mlp(P, seed=1)
    p = (np.random.default_rng(seed).standard_normal(net.n_params) * scale).astype(np.float32)
    net.set_params(p)
    return net, p


def test_bf16_copy_is_round_to_nearest_even():
    net, p = _net()
    master, bits = net.params()
    assert (master == p).all()
    assert (bits == om.bf16_bits(p)).all()
    net.close()


def test_fresh_net_is_near_geometric():
    net = pt.Mlp(P, seed=3)
    x, _ = _rows(np.random.default_rng(0), 8)
    z = net.forward(x)
    f = om.shape_fractions(z.astype(np.float64), P)
    assert np.abs(f * P - 1).max() < 0.05
    net.close()


def test_forward_matches_oracle():
    net, p = _net()
    x, _ = _rows(np.random.default_rng(1), B)
    z = net.forward(x)
    zr, _ = om.forward(om.bf16_params(p, P), x, P)
    assert np.abs(z - zr).max() <= 2e-6 * max(1.0, np.abs(zr).max())
    net.close()


@pytest.mark.parametrize("w_kappa", [0.0, 1.0, 4.0])
def test_loss_and_gradient_match_oracle(w_kappa):
    net, p = _net(seed=7)
    x, t = _rows(np.random.default_rng(2), B)
    loss, g = net.loss_grad(x, t, w_kappa)
    Lr, gr = om.loss_grad(om.bf16_params(p, P), x, t, P, w_kappa)
    assert loss == pytest.approx(Lr, rel=2e-5)
    # gradient through the bfloat16 weights: float accumulation only
    assert np.linalg.norm(g - gr) <= 1e-4 * np.linalg.norm(gr)
    assert np.abs(g - gr).max() <= 1e-4 * np.abs(gr).max()
    # against the exact gradient at the float master weights: bfloat16 error
    _, g32 = om.loss_grad(p.astype(np.float64), x, t, P, w_kappa)
    assert np.linalg.norm(g - g32) <= 1e-2 * np.linalg.norm(g32)
    net.close()


def test_adam_steps_match_oracle():
    net, p = _net(seed=9)
    x, t = _rows(np.random.default_rng(3), B)
    ref = p.astype(np.float64)
    m = v = np.zeros_like(ref)
    lr = 3e-3
    for step in range(1, 4):
        _, g = net.loss_grad(x, t, 1.0)
        net.train(x, t, 1, lr=lr, w_kappa=1.0)
        got, bits = net.params()
        ref, m, v = om.adam_step(ref, m, v, g.astype(np.float64), step, lr)
        assert np.abs(got - ref).max() <= 1e-6 * max(1.0, np.abs(ref).max())
        assert (bits == om.bf16_bits(got)).all()
        ref = got.astype(np.float64)  # continue from the device's float state
    net.close()


def test_ladder_decoding_matches_oracle():
    net, p = _net(seed=11, scale=0.4)
    rng = np.random.default_rng(4)
    n = 37
    x, _ = _rows(rng, n)
    bmin = rng.uniform(0.5, 3.0, n)
    bmax = bmin * rng.uniform(1.2, 5.0, n)
    nt = rng.choice([2, 3, 5, 16, 17, 33, 48, 78], n).astype(np.int32)
    out = net.ladder(x, bmin, bmax, nt, 2.0)
    z = net.forward(x).astype(np.float64)
    # rows that let the net choose the replica count
    sig = 1.7
    nt_free = np.where(np.arange(n) % 3 == 0, 0, nt)
    free = net.ladder(x, bmin, bmax, nt_free, 2.0, sigma_target=sig, max_temps=96)
    for r in range(n):
        want = om.replica_count(z[r], P, sig, 96) if nt_free[r] == 0 else nt[r]
        assert free[r][0].shape == (want,)
        np.testing.assert_allclose(free[r][0], om.decode(z[r], P, bmin[r], bmax[r], want, 2.0)[0], rtol=1e-6)
    for r in range(n):
        b, e = out[r]
        br, er = om.decode(z[r], P, bmin[r], bmax[r], nt[r], 2.0)
        assert b.shape == (nt[r],) and e.shape == (nt[r] - 1,)
        assert b[0] == bmin[r] and b[-1] == bmax[r]
        assert (np.diff(b) > 0).all()
        np.testing.assert_allclose(b, br, rtol=1e-6)
        np.testing.assert_allclose(e, er, rtol=1e-5, atol=1e-9)
    net.close()


def test_ladder_rejects_bad_ranges():
    net = pt.Mlp(P, seed=1)
    x = np.zeros((1, 4), np.float32)
    for bmin, bmax, nt in ((2.0, 2.0, 4), (0.0, 2.0, 4), (2.0, 3.0, 1)):
        with pytest.raises(pt.PtError):
            net.ladder(x, bmin, bmax, nt, 1.0)
    net.close()


def _smooth_targets(x, P=P):
    """A smooth synthetic map features -> (shape, kappa curve)."""
    u = (np.arange(P) + 0.5) / P
    a = 0.8 * (x[:, 0:1] - 2.5) + 0.3 * (x[:, 1:2] - 2.0)
    f = np.exp(a * (u[None] - 0.5))
    f /= f.sum(1, keepdims=True)
    e = 0.25 + 0.1 * np.tanh((x[:, 2:3] - 7.0)) * (u[None] - 0.5)
    lam = 1.5 * x[:, 0:1] + np.log(np.log(x[:, 2:3] / x[:, 1:2])) - 1.0
    return np.concatenate([f, e, lam], axis=1).astype(np.float32)


def test_training_converges_and_is_deterministic():
    rng = np.random.default_rng(6)
    x, _ = _rows(rng, 200)
    t = _smooth_targets(x)
    nets = [pt.Mlp(P, seed=21) for _ in range(2)]
    losses = nets[0].train(x, t, 1500, lr=2e-3, record=True)
    nets[1].train(x, t, 1500, lr=2e-3)
    assert losses[-1] < 0.02 * losses[0]
    p0, _ = nets[0].params()
    p1, _ = nets[1].params()
    assert (p0 == p1).all()
    # held-out rows from the same map
    xv, _ = _rows(np.random.default_rng(60), 50)
    zv = nets[0].forward(xv).astype(np.float64)
    fv = om.shape_fractions(zv, P)
    tv = _smooth_targets(xv)
    assert np.abs(fv * P - tv[:, :P] * P).max() < 0.1
    assert np.abs(zv[:, 2 * P] - tv[:, 2 * P]).mean() < 0.05
    assert np.abs(zv[:, 2 * P] - tv[:, 2 * P]).max() < 0.3
    for n in nets:
        n.close()
