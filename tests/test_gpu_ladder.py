"""What the trained ladder network gains over the method without it.

The network is trained on the device by the pt_mlp_* kernels from the
shipped training set (acceptances the engine measured in kappa scans on
geometric ladders, ``paper_1006_4247_gb300/data/ladder_train.npz``) and
evaluated on held-out coupling samples at a lattice size it never saw
(L = 10), inverse temperatures 2..8, against:

* the yardstick: the geometric ladder with one cooling/heating parameter for
  all pairs, tuned by a scan on the evaluation samples themselves (the
  paper's procedure, section III.B), at the replica count of the paper's rule;
* the same geometric ladder with epsilon tuned per pair and per sample from
  that scan (no network: the ablation of the learned parameters);
* the plain swap on the same geometric ladder (the standard method).

All arms run as samples of one batched engine (cooling/heating exchange,
1 heat-bath + 5L/4 overrelaxation sweeps per cycle); acceptance per pair and
round trips per chain are counted after a burn-in.  The summary is printed
(run with -s).
"""
import json

import numpy as np
import pytest

from paper_1006_4247_gb300 import ladder as lad
from paper_1006_4247_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EVAL_L = 10
WINDOW = (2.0, 8.0)
N_SAMPLES = 8
CYCLES, BURN = 20000, 2000


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1006_4247_gb300 import _build
    _build.build()


@pytest.fixture(scope="module")
def trained():
    d = np.load(lad.TRAIN_FILE)
    net, losses = lad.train(d["X"], d["T"], steps=4000)
    yield net, losses
    net.close()


def test_training_on_device_reduces_loss_and_reproduces_shipped_net(trained):
    net, losses = trained
    assert np.isfinite(losses).all()
    assert losses[-1] < 0.1 * losses[0]
    p, _ = net.net.params()
    shipped = np.load(lad.WEIGHTS_FILE)["params"]
    assert p.shape == shipped.shape
    assert np.abs(p - shipped).max() <= 1e-3 * max(1.0, np.abs(shipped).max())


def _summary(res):
    """Per sample: worst pair, mean and relative spread of the acceptance;
    round trips per chain (both copies).  Means and errors over samples."""
    amin = np.array([a.min() for a, _ in res])
    amean = np.array([a.mean() for a, _ in res])
    spread = np.array([(a.max() - a.min()) / a.mean() for a, _ in res])
    rt = np.array([r.sum() / 2 for _, r in res])
    return {"rt_per_chain": float(rt.mean()), "rt_se": float(rt.std(ddof=1) / np.sqrt(len(rt))),
            "acc_min": float(amin.mean()), "acc_mean": float(amean.mean()), "acc_spread": float(spread.mean())}


def test_learned_ladder_against_geometric(trained):
    net, _ = trained
    samples = [(EVAL_L, W.couplings(EVAL_L, 7000 + k), *WINDOW) for k in range(N_SAMPLES)]
    NT = lad.default_n_temps(EVAL_L, *WINDOW)
    geo = lad.geometric(*WINDOW, NT)
    # the yardstick's kappa: a scan on the evaluation samples themselves
    scan = [(L, J, geo, lad.eps_from_kappa(geo, np.full(NT - 1, k), lad.eps_bound(L, J)))
            for k in lad.KAPPA_GRID for (L, J, _, _) in samples]
    res = lad.run_ladders(scan, 2000, 1000, seed=41)
    acc_k = np.array([np.mean([res[i * N_SAMPLES + s][0].mean() for s in range(N_SAMPLES)])
                      for i in range(len(lad.KAPPA_GRID))])
    kappa = lad.KAPPA_GRID[int(np.argmax(acc_k))]
    geo_min = float(np.mean([res[int(np.argmax(acc_k)) * N_SAMPLES + s][0].min() for s in range(N_SAMPLES)]))
    # per-pair kappa of each sample from the same scan
    per_pair = []
    for k_, (L, J, _, _) in enumerate(samples):
        acc_s = np.stack([res[i * N_SAMPLES + k_][0] for i in range(len(lad.KAPPA_GRID))])
        kb, _ = lad.best_kappa(lad.KAPPA_GRID, acc_s)
        per_pair.append(lad.eps_from_kappa(geo, kb, lad.eps_bound(L, J)))

    learned = net.propose_many(samples, n_temps=NT)
    auto = net.propose_many(samples, target_acceptance=geo_min)
    nt_small = int(round(0.7 * NT))
    small = net.propose_many(samples, n_temps=nt_small)
    arms = {"geometric": [], "geometric_per_pair": [], "learned": [], "learned_auto": [], "learned_small": []}
    cases = []
    for k, (L, J, _, _) in enumerate(samples):
        b, e = lad.geometric_reference(L, J, *WINDOW, NT, kappa)
        cases.append((L, J, b, e)); arms["geometric"].append(len(cases) - 1)
        cases.append((L, J, geo, per_pair[k])); arms["geometric_per_pair"].append(len(cases) - 1)
        cases.append((L, J, *learned[k])); arms["learned"].append(len(cases) - 1)
        cases.append((L, J, *auto[k])); arms["learned_auto"].append(len(cases) - 1)
        cases.append((L, J, *small[k])); arms["learned_small"].append(len(cases) - 1)
    res = lad.run_ladders(cases, CYCLES, BURN, seed=43)
    plain = lad.run_ladders([(L, J, geo, np.zeros(NT - 1, np.float32)) for (L, J, _, _) in samples],
                            CYCLES, BURN, seed=43, mode="plain")
    out = {name: _summary([res[i] for i in idx]) for name, idx in arms.items()}
    out["plain_geometric"] = _summary(plain)
    out["n_temps"] = {"geometric": NT, "geometric_per_pair": NT, "learned": NT, "learned_auto": [len(a[0]) for a in auto],
                      "learned_small": nt_small, "plain_geometric": NT}
    out["kappa_scan"] = {"grid": list(lad.KAPPA_GRID), "acc_mean": acc_k.round(4).tolist(), "chosen": kappa}
    out["learned_kappa"] = [float(np.mean(e / np.diff(np.log(b)))) for b, e in learned]
    print("\nlearned ladder vs geometric:", json.dumps(out))

    g, l = out["geometric"], out["learned"]
    # the net's epsilons do as well as the scan-tuned one, without a scan
    assert l["acc_mean"] >= 0.95 * g["acc_mean"]
    # equalised acceptance: flatter profile, higher worst pair
    assert l["acc_spread"] < g["acc_spread"]
    assert l["acc_min"] >= g["acc_min"]
    # round trips not worse than the yardstick's within the noise
    assert l["rt_per_chain"] >= g["rt_per_chain"] - 3 * np.hypot(l["rt_se"], g["rt_se"])
    # fewer replicas for the yardstick's worst-pair acceptance
    assert max(out["n_temps"]["learned_auto"]) <= NT
    # learned ladder + modified exchange: the plain method's round-trip rate with 30% fewer replicas
    assert out["learned_small"]["rt_per_chain"] >= out["plain_geometric"]["rt_per_chain"]


def test_feedback_controller_reaches_scan_tuned_acceptance():
    """Per-pair epsilon tuned online from the measured acceptance, with no
    network and no scan (the ablation of the network's epsilon): started at
    the low end of the scan grid, ten iterations of a sign controller reach
    the acceptance of the scan-tuned kappa on the held-out samples."""
    samples = [(EVAL_L, W.couplings(EVAL_L, 7000 + k)) for k in range(N_SAMPLES)]
    NT = lad.default_n_temps(EVAL_L, *WINDOW)
    geo = lad.geometric(*WINDOW, NT)
    kap, hist, spent = lad.feedback_kappa([(L, J, geo) for L, J in samples], kappa0=lad.KAPPA_GRID[0], seed=51)
    cases = []
    for L, J in samples:
        bd = lad.eps_bound(L, J)
        cases += [(L, J, geo, lad.eps_from_kappa(geo, np.full(NT - 1, k), bd)) for k in lad.KAPPA_GRID]
    for (L, J), k in zip(samples, kap):
        cases.append((L, J, geo, lad.eps_from_kappa(geo, k, lad.eps_bound(L, J))))
    res = lad.run_ladders(cases, 4000, 1000, seed=53)
    nk = len(lad.KAPPA_GRID)
    grid_acc = np.array([[res[s * nk + i][0].mean() for i in range(nk)] for s in range(N_SAMPLES)])  # [S, K]
    best = int(np.argmax(grid_acc.mean(0)))
    fb = np.array([res[N_SAMPLES * nk + s][0].mean() for s in range(N_SAMPLES)])
    fb_min = np.array([res[N_SAMPLES * nk + s][0].min() for s in range(N_SAMPLES)])
    scan_min = np.array([res[s * nk + best][0].min() for s in range(N_SAMPLES)])
    out = {"kappa_grid": list(lad.KAPPA_GRID), "grid_acc": grid_acc.mean(0).round(4).tolist(),
           "scan_kappa": lad.KAPPA_GRID[best], "feedback_kappa_mean": float(np.mean([k.mean() for k in kap])),
           "feedback_acc": float(fb.mean()), "feedback_worst_pair": float(fb_min.mean()),
           "scan_worst_pair": float(scan_min.mean()), "history": [round(h, 4) for h in hist],
           "tuning_cycles": spent}
    print("\nfeedback controller:", json.dumps(out))
    assert fb.mean() >= 0.98 * grid_acc.mean(0)[best]        # the scan's acceptance without the scan
    assert fb.mean() > grid_acc.mean(0)[0] + 0.01              # clearly above where it started
    assert fb_min.mean() >= 0.95 * scan_min.mean()
    assert hist[-1] > hist[0]
