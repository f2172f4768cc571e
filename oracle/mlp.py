"""Plain FP64 oracle of the learned ladder network (numpy).

TEST INFRASTRUCTURE ONLY: the test-suite may import this module; the engine
in ``paper_1006_4247_gb300`` never does, and it shares no code with the CUDA
kernels.

The network and its decoding are this project's design (the paper has no
network); the decoding serves the paper's tempering parameters: the ladder of
inverse temperatures beta_i and the cooling/heating parameter epsilon of every
pair (section III.B, whose optimal value depends on the pair and falls with
beta_{i+1}/beta_i).  Everything is written out as its definition, in double
precision, one operation at a time:

  perceptron  h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), z = W3 h2 + b3
  shape       d_k = softplus(z_k) + 0.01, f_k = d_k / sum_j d_j, k < P
  loss        (1/P) sum_k (P (f_k - t_k))^2 + w (sigmoid(z_{P+k}) - t_{P+k})^2
              + (z_{2P} - t_{2P})^2, averaged over rows
  gradient    reverse-mode differentiation of the above, written by hand
  Adam        Kingma & Ba (2015), Algorithm 1, bias-corrected
  bfloat16    round-to-nearest-even of the float32 bit pattern to its upper
              16 bits (the format's definition)
  decode      ln beta(u) = ln beta_min + F(u) ln(beta_max / beta_min),
              F piecewise linear through the knots (k / P, sum_{j<k} f_j);
              eps_i = kappa_max e(midpoint) (ln beta_{i+1} - ln beta_i), e
              piecewise linear through (k + 1/2) / P, flat beyond the ends;
              replica count NT = 1 + ceil(exp(z_{2P}) / sigma_target)

Parity status (tests/test_oracle_mlp.py): forward pinned by a hand-computed
network; gradient pinned by central finite differences of the loss; Adam by
its closed-form first step; bfloat16 rounding by hand-made bit patterns and
by torch's conversion; decode by the geometric closed form (equal shape
outputs), end points, monotonicity and the constant-kappa closed form.
"""
from __future__ import annotations

import numpy as np

IN, HID = 4, 64
SHAPE_FLOOR = np.float32(0.01).astype(np.float64)  # the float constant of the kernels


def layout(P: int) -> dict:
    """Offsets of [W1 | b1 | W2 | b2 | W3 | b3] in the flat parameter vector."""
    N = 2 * P + 1
    o = {}
    off = 0
    for name, size in (("W1", HID * IN), ("b1", HID), ("W2", HID * HID), ("b2", HID),
                       ("W3", N * HID), ("b3", N)):
        o[name] = (off, size)
        off += size
    o["total"] = off
    return o


def unpack(params, P):
    lay = layout(P)
    p = np.asarray(params, np.float64)
    get = lambda k: p[lay[k][0]:lay[k][0] + lay[k][1]]
    return (get("W1").reshape(HID, IN), get("b1"), get("W2").reshape(HID, HID), get("b2"),
            get("W3").reshape(2 * P + 1, HID), get("b3"))


def pack(W1, b1, W2, b2, W3, b3):
    return np.concatenate([np.ravel(a) for a in (W1, b1, W2, b2, W3, b3)]).astype(np.float64)


def softplus(z):
    z = np.asarray(z, np.float64)
    return np.where(z > 30.0, z, np.log1p(np.exp(np.minimum(z, 30.0))))


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-np.asarray(z, np.float64)))


def forward(params, x, P):
    """z [B, 2P] and the hidden activations (h1, h2)."""
    W1, b1, W2, b2, W3, b3 = unpack(params, P)
    x = np.asarray(x, np.float64)
    h1 = np.maximum(x @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    z = h2 @ W3.T + b3
    return z, (h1, h2)


def shape_fractions(z, P):
    d = softplus(z[:, :P]) + SHAPE_FLOOR
    return d / d.sum(axis=1, keepdims=True)


def loss(params, x, t, P, w_kappa):
    z, _ = forward(params, x, P)
    t = np.asarray(t, np.float64)
    f = shape_fractions(z, P)
    e = sigmoid(z[:, P:2 * P])
    row = ((P * (f - t[:, :P])) ** 2).sum(1) + w_kappa * ((e - t[:, P:2 * P]) ** 2).sum(1)
    return float((row / P + (z[:, 2 * P] - t[:, 2 * P]) ** 2).mean())


def loss_grad(params, x, t, P, w_kappa):
    """(loss, dloss/dparams) by hand-written reverse-mode differentiation."""
    W1, b1, W2, b2, W3, b3 = unpack(params, P)
    x = np.asarray(x, np.float64)
    t = np.asarray(t, np.float64)
    B = x.shape[0]
    z, (h1, h2) = forward(params, x, P)
    d = softplus(z[:, :P]) + SHAPE_FLOOR
    S = d.sum(1, keepdims=True)
    f = d / S
    e = sigmoid(z[:, P:2 * P])
    dl = z[:, 2 * P] - t[:, 2 * P]
    row = ((P * (f - t[:, :P])) ** 2).sum(1) + w_kappa * ((e - t[:, P:2 * P]) ** 2).sum(1)
    L = float((row / P + dl ** 2).mean())
    # dL/df and dL/de, with the 1/(P B) of the means
    df = 2.0 * P * P * (f - t[:, :P]) / (P * B)
    de = 2.0 * w_kappa * (e - t[:, P:2 * P]) / (P * B)
    # f_k = d_k / S: dL/dd_j = dL/df_j / S - sum_k dL/df_k d_k / S^2
    dd = df / S - (df * d).sum(1, keepdims=True) / S ** 2
    gz = np.concatenate([dd * sigmoid(z[:, :P]), de * e * (1.0 - e), (2.0 * dl / B)[:, None]], axis=1)
    gW3 = gz.T @ h2
    gb3 = gz.sum(0)
    gh2 = (gz @ W3) * (h2 > 0)
    gW2 = gh2.T @ h1
    gb2 = gh2.sum(0)
    gh1 = (gh2 @ W2) * (h1 > 0)
    gW1 = gh1.T @ x
    gb1 = gh1.sum(0)
    return L, pack(gW1, gb1, gW2, gb2, gW3, gb3)


def adam_step(params, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """Step t (1-based) of Adam: returns (params, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_bits(a):
    """bfloat16 bit patterns of float32 values, round to nearest, ties to
    even (finite inputs)."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    lower = u & 0xFFFF
    upper = u >> 16
    round_up = (lower > 0x8000) | ((lower == 0x8000) & ((upper & 1) == 1))
    return ((upper + round_up) & 0xFFFF).astype(np.uint16)


def bf16_value(bits):
    """float64 value of bfloat16 bit patterns."""
    return (np.asarray(bits, np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def bf16_params(params, P):
    """The parameter vector as the products see it: weights rounded to
    bfloat16, biases exact (float32)."""
    lay = layout(P)
    p32 = np.asarray(params, np.float32)
    out = p32.astype(np.float64)
    for k in ("W1", "W2", "W3"):
        a, n = lay[k]
        out[a:a + n] = bf16_value(bf16_bits(p32[a:a + n]))
    return out


def replica_count(z, P, sigma_target, max_temps):
    """NT = 1 + ceil(Lambda / sigma_target), Lambda = exp(z_{2P}), in [2, max_temps]."""
    nt = 1.0 + np.ceil(np.exp(np.float64(z[2 * P])) / sigma_target)
    return int(min(max(nt, 2.0), max_temps))


def decode(z, P, beta_min, beta_max, n_temps, kappa_max):
    """Ladder (betas [NT]) and epsilons ([NT - 1]) of one row of outputs."""
    z = np.asarray(z, np.float64)
    d = softplus(z[:P]) + SHAPE_FLOOR
    f = d / d.sum()
    F = np.concatenate([[0.0], np.cumsum(f)])
    F[-1] = 1.0
    e = sigmoid(z[P:2 * P])
    lb0, lb1 = np.log(beta_min), np.log(beta_max)
    NT = int(n_temps)
    lnb = np.empty(NT)
    for i in range(NT):
        u = i / (NT - 1)
        Fu = np.interp(u, np.arange(P + 1) / P, F)
        lnb[i] = lb0 + (lb1 - lb0) * Fu
    lnb[0], lnb[-1] = lb0, lb1
    betas = np.exp(lnb)
    betas[0], betas[-1] = beta_min, beta_max
    mids = (np.arange(NT - 1) + 0.5) / (NT - 1)
    ev = np.interp(mids, (np.arange(P) + 0.5) / P, e)  # flat beyond the outer midpoints
    eps = kappa_max * ev * np.diff(lnb)
    return betas, eps
