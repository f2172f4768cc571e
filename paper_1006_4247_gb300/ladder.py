"""Learned inverse-temperature ladder and per-pair cooling/heating parameter.

The paper tempers with a geometric ladder of temperatures (section IV) and one
cooling/heating parameter epsilon for all pairs (section III.B), which it notes
should depend on the pair and fall with beta_{i+1}/beta_i.  This module
replaces both choices by the proposals of a small network (``pt.Mlp``, the
pt_mlp_* kernels), trained on data the engine itself produces:

* a scan runs the cooling/heating exchange on a geometric ladder with a few
  values of kappa = eps / ln(beta_{i+1}/beta_i) per sample and records the
  acceptance of every pair;
* per pair, the best kappa and its acceptance give the target parameter
  curve kappa(beta) and the local "rejection density" per unit of ln beta;
  equal spacing in that density equalises the acceptance along the ladder
  and gives the target shape F(u);
* the network maps the features of a sample to (shape, kappa curve); it is
  trained on the device by the project's own forward/backward/Adam kernels.

The Markov chain stays exact for every ladder and every epsilon: the network
only chooses parameters of the tempering.  The geometric ladder with one
tuned kappa is the fallback and the yardstick (round trips per chain, lowest
pair acceptance).

All functions run on the host except the engine and network calls, which go
through the C ABI (no CPU fallback).
"""
from __future__ import annotations

import argparse
import dataclasses
import math
import os

import numpy as np

from . import pt
from . import workloads

N_KNOTS = 16
KAPPA_MAX = 0.5
KAPPA_GRID = (0.04, 0.07, 0.1, 0.13, 0.17, 0.22)
DATA_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")
TRAIN_FILE = os.path.join(DATA_DIR, "ladder_train.npz")
WEIGHTS_FILE = os.path.join(DATA_DIR, "ladder_net.npz")
PAPER_WINDOW = (1 / 0.19, 1 / 0.12)  # section IV: T from 0.12 to 0.19
TRAIN_L = (4, 6, 8, 12, 16, 24, 32)
TRAIN_WINDOWS = ((2.0, 8.0), (2.5, 8.0), PAPER_WINDOW, (3.0, 6.0), (4.0, 10.0), (1.5, 5.0))
EPS_SAFETY = 0.9  # eps * max_x sum_6 |J| must stay below 1 (invertible cooling step)


# ---------------------------------------------------------------- features
def coupling_statistic(L: int, J: np.ndarray) -> float:
    """g = mean_x sqrt(sum_{y nn x} J_xy^2) / (sqrt(6) rms J): the typical
    local-field scale of the sample in units of its coupling width (about
    0.96 for Gaussian couplings)."""
    J = np.asarray(J, np.float64).reshape(3, L, L, L)
    sq = np.zeros((L, L, L))
    for mu in range(3):
        a = J[mu] ** 2
        sq += a + np.roll(a, 1, axis=2 - mu)
    rms = math.sqrt(float((J ** 2).mean()))
    return float(np.sqrt(sq).mean() / (math.sqrt(6.0) * rms))


def features(L: int, J: np.ndarray, beta_min: float, beta_max: float) -> np.ndarray:
    """The network's input: (ln L, beta_min, beta_max, g)."""
    return np.array([math.log(L), beta_min, beta_max, coupling_statistic(L, J)], np.float32)


def eps_bound(L: int, J: np.ndarray) -> float:
    """Largest epsilon kept: EPS_SAFETY / max_x sum_6 |J_xy|."""
    A = np.abs(np.asarray(J, np.float64)).reshape(3, L, L, L)
    s = np.zeros((L, L, L))
    for mu in range(3):
        s += A[mu] + np.roll(A[mu], 1, axis=2 - mu)
    return EPS_SAFETY / float(s.max())


def geometric(beta_min: float, beta_max: float, n_temps: int) -> np.ndarray:
    """Geometric ladder (section IV): equal ratios beta_{i+1}/beta_i."""
    return beta_min * (beta_max / beta_min) ** (np.arange(n_temps) / (n_temps - 1))


def eps_from_kappa(betas: np.ndarray, kappa, bound: float) -> np.ndarray:
    """eps_i = kappa_i ln(beta_{i+1}/beta_i), capped at the invertibility bound."""
    e = np.asarray(kappa, np.float64) * np.diff(np.log(betas))
    return np.minimum(e, bound).astype(np.float32)


def default_n_temps(L: int, beta_min: float, beta_max: float) -> int:
    """Replica count of the geometric reference ladder: N_T - 1 proportional
    to L^{3/2} ln(beta_max/beta_min), the constant fixed by the paper's
    ladders (section IV: T in [0.12, 0.19] with N_T = 15 at L = 16 and 27 at
    L = 24)."""
    return max(3, 1 + int(round(0.48 * L ** 1.5 * math.log(beta_max / beta_min))))


# ---------------------------------------------------------------- targets
def sigma_of_acceptance(acc):
    """Width of the Gaussian log-acceptance-ratio that gives acceptance a:
    a = erfc(sigma / (2 sqrt 2)) for ln A ~ N(-sigma^2/2, sigma^2)."""
    from scipy.special import erfcinv
    a = np.clip(np.asarray(acc, np.float64), 0.005, 0.995)
    return 2.0 * math.sqrt(2.0) * erfcinv(a)


def acceptance_of_sigma(sigma):
    from scipy.special import erfc
    return erfc(np.asarray(sigma, np.float64) / (2.0 * math.sqrt(2.0)))


def equal_acceptance_shape(betas: np.ndarray, acc: np.ndarray, P: int = N_KNOTS) -> np.ndarray:
    """Shape fractions f_k (k < P, summing to 1) of the ladder that spaces
    the replicas equally in the cumulative rejection density
    Lambda(ln beta) = int sigma / d(ln beta), interpolated from the
    acceptance of the measured ladder."""
    lnb = np.log(np.asarray(betas, np.float64))
    lam = sigma_of_acceptance(acc)  # per interval
    cum = np.concatenate([[0.0], np.cumsum(lam)])
    u = np.arange(P + 1) / P
    target_ln = np.interp(u * cum[-1], cum, lnb)
    F = (target_ln - lnb[0]) / (lnb[-1] - lnb[0])
    F[0], F[-1] = 0.0, 1.0
    return np.maximum(np.diff(F), 1e-6) / np.maximum(np.diff(F), 1e-6).sum()


def shape_ladder(beta_min, beta_max, f, n_temps):
    """Ladder of a shape: ln beta(u) = ln beta_min + F(u) ln(beta_max/beta_min)."""
    P = len(f)
    F = np.concatenate([[0.0], np.cumsum(f)])
    F[-1] = 1.0
    u = np.arange(n_temps) / (n_temps - 1)
    lb = math.log(beta_min) + np.interp(u, np.arange(P + 1) / P, F) * math.log(beta_max / beta_min)
    b = np.exp(lb)
    b[0], b[-1] = beta_min, beta_max
    return b


def best_kappa(kappas, acc_by_kappa):
    """Per pair, the kappa of highest acceptance (parabola through the best
    grid point and its neighbours, kept inside the grid) and that acceptance.
    acc_by_kappa: [n_kappa, n_pairs]."""
    k = np.asarray(kappas, np.float64)
    A = np.asarray(acc_by_kappa, np.float64)
    best = np.empty(A.shape[1])
    amax = A.max(0)
    for i in range(A.shape[1]):
        j = int(np.argmax(A[:, i]))
        if 0 < j < len(k) - 1:
            x, y = k[j - 1:j + 2], A[j - 1:j + 2, i]
            c2, c1, _ = np.polyfit(x, y, 2)
            best[i] = float(np.clip(-c1 / (2 * c2), x[0], x[2])) if c2 < 0 else k[j]
        else:
            best[i] = k[j]
    return best, amax


# ---------------------------------------------------------------- engine runs
@dataclasses.dataclass
class Row:
    """One training case: a coupling sample and an inverse-temperature range."""
    L: int
    J: np.ndarray          # float32 [3, L^3]
    beta_min: float
    beta_max: float
    n_temps: int = 0

    def __post_init__(self):
        if not self.n_temps:
            self.n_temps = default_n_temps(self.L, self.beta_min, self.beta_max)


def run_ladders(cases, n_cycles, n_burn, seed=0, mode="coolheat", n_copies=2):
    """Run each case (L, J, betas, eps) as one sample of a single batched
    engine: n_burn + n_cycles update cycles (1 heat-bath + 5L/4
    overrelaxation sweeps per sample + one tempering update).  Returns per
    case (acceptance per pair [n_copies, NT-1] pooled over copies as [NT-1],
    round trips per chain [n_copies]), counted over the last n_cycles."""
    Ls = [c[0] for c in cases]
    Js = [np.asarray(c[1], np.float32) for c in cases]
    Bs = [np.asarray(c[2], np.float64) for c in cases]
    eps = np.concatenate([np.asarray(c[3], np.float32) for c in cases])
    n_or = np.array([max(1, (5 * L) // 4) for L in Ls], np.int32)
    eng = pt.Engine(Ls, Js, Bs, n_copies=n_copies, seed=seed)
    try:
        eng.set_params(None, eps)
        eng.cycles(n_burn, 1, int(n_or.max()), mode, n_or_samples=n_or)
        p0, a0, r0, _ = eng.stats()
        eng.cycles(n_cycles, 1, int(n_or.max()), mode, n_or_samples=n_or)
        p1, a1, r1, _ = eng.stats()
    finally:
        eng.close()
    out = []
    off = 0
    for s, B in enumerate(Bs):
        n = n_copies * (len(B) - 1)
        prop = (p1 - p0)[off:off + n].reshape(n_copies, -1).sum(0)
        acc = (a1 - a0)[off:off + n].reshape(n_copies, -1).sum(0)
        off += n
        rt = (r1 - r0)[s * n_copies:(s + 1) * n_copies]
        out.append((acc / np.maximum(prop, 1), rt))
    return out


def feedback_kappa(cases, n_iter=10, block=300, kappa0=0.07, delta=0.35, step0=0.4, decay=0.75, n_burn=500,
                   seed=0, mode="coolheat", n_copies=2, kappa_min=0.005):
    """Per-pair cooling parameter by feedback on the measured acceptance, with
    neither the network nor a scan (the paper notes that epsilon should
    depend on the pair, sections III.B and IV.A).  Each case is (L, J, betas).

    kappa_i = eps_i / ln(beta_{i+1}/beta_i) is tuned on a log scale.  The
    chain is exact for every epsilon and the proposals of pair i depend on
    eps_i alone, so all pairs of all samples are tuned at once in one
    batched engine without re-equilibrating between settings: every
    iteration runs `block` cycles with every ln kappa_i raised by `delta`
    and `block` cycles with it lowered by `delta`, then moves ln kappa_i by
    the current step towards the side whose acceptance (pooled over the
    copies) was higher; the step shrinks by `decay` per iteration.
    Returns (kappa per case [NT-1], history of the mean acceptance per
    iteration, cycles spent)."""
    Ls = [c[0] for c in cases]
    Js = [np.asarray(c[1], np.float32) for c in cases]
    Bs = [np.asarray(c[2], np.float64) for c in cases]
    bounds = [eps_bound(L, J) for L, J in zip(Ls, Js)]
    u = [np.full(len(B) - 1, math.log(kappa0)) for B in Bs]
    n_or = np.array([max(1, (5 * L) // 4) for L in Ls], np.int32)
    lo, hi = math.log(kappa_min), math.log(KAPPA_MAX)

    def eps_of(shift):
        return np.concatenate([eps_from_kappa(B, np.exp(np.clip(uu + shift, lo, hi)), bd)
                               for B, uu, bd in zip(Bs, u, bounds)])

    eng = pt.Engine(Ls, Js, Bs, n_copies=n_copies, seed=seed)
    spent = 0

    def block_acc(eps, n):
        nonlocal spent
        eng.set_params(None, eps)
        p0, a0, _, _ = eng.stats()
        eng.cycles(n, 1, int(n_or.max()), mode, n_or_samples=n_or)
        p1, a1, _, _ = eng.stats()
        spent += n
        out, off = [], 0
        for B in Bs:
            m = n_copies * (len(B) - 1)
            prop = (p1 - p0)[off:off + m].reshape(n_copies, -1).sum(0)
            acc = (a1 - a0)[off:off + m].reshape(n_copies, -1).sum(0)
            off += m
            out.append(acc / np.maximum(prop, 1))
        return out

    hist = []
    try:
        block_acc(eps_of(0.0), n_burn)
        step = step0
        for _ in range(n_iter):
            ap = block_acc(eps_of(+delta), block)
            am = block_acc(eps_of(-delta), block)
            for k in range(len(u)):
                u[k] = np.clip(u[k] + step * np.sign(ap[k] - am[k]), lo, hi)
            hist.append(float(np.mean([0.5 * (a + b).mean() for a, b in zip(ap, am)])))
            step *= decay
    finally:
        eng.close()
    return [np.exp(uu) for uu in u], hist, spent


def training_targets(rows, n_cycles=1500, n_burn=500, seed=0, kappas=KAPPA_GRID, P=N_KNOTS):
    """Scan kappa on the geometric ladder of every row and derive its targets.
    Returns (features [B, 4], targets [B, 2P+1], info) with targets
    [shape fractions | kappa / KAPPA_MAX | ln Lambda], Lambda the sum over
    the pairs of sigma at the best kappa."""
    cases = []
    for r in rows:
        b = geometric(r.beta_min, r.beta_max, r.n_temps)
        bound = eps_bound(r.L, r.J)
        for k in kappas:
            cases.append((r.L, r.J, b, eps_from_kappa(b, np.full(r.n_temps - 1, k), bound)))
    res = run_ladders(cases, n_cycles, n_burn, seed=seed)
    X, T, info = [], [], []
    nk = len(kappas)
    for i, r in enumerate(rows):
        acc = np.stack([res[i * nk + j][0] for j in range(nk)])
        kbest, abest = best_kappa(kappas, acc)
        b = geometric(r.beta_min, r.beta_max, r.n_temps)
        f = equal_acceptance_shape(b, abest, P)
        # kappa target at the knot midpoints of the target ladder
        lnb = np.log(b)
        mids_ln = 0.5 * (lnb[1:] + lnb[:-1])
        F = np.concatenate([[0.0], np.cumsum(f)])
        um = (np.arange(P) + 0.5) / P
        ln_at = lnb[0] + np.interp(um, np.arange(P + 1) / P, F) * (lnb[-1] - lnb[0])
        kap = np.interp(ln_at, mids_ln, kbest)
        X.append(features(r.L, r.J, r.beta_min, r.beta_max))
        lam_total = float(sigma_of_acceptance(abest).sum())
        T.append(np.concatenate([f, np.clip(kap / KAPPA_MAX, 0.01, 0.99), [math.log(lam_total)]]))
        info.append({"acc": acc, "kappa_best": kbest, "acc_best": abest})
    return np.stack(X).astype(np.float32), np.stack(T).astype(np.float32), info


# ---------------------------------------------------------------- proposals
class LearnedLadder:
    """The trained network and its proposals (betas, eps) per sample."""

    def __init__(self, n_knots=N_KNOTS, seed=1, stream=None):
        self.net = pt.Mlp(n_knots, seed=seed, stream=stream)

    def train(self, X, T, steps=3000, lr=2e-3, w_kappa=1.0, record=False):
        return self.net.train(X, T, steps, lr=lr, w_kappa=w_kappa, record=record)

    @classmethod
    def load(cls, path=WEIGHTS_FILE, stream=None):
        """The shipped (or a saved) trained net."""
        d = np.load(path)
        self = cls(int(d["n_knots"]), stream=stream)
        self.net.set_params(d["params"])
        return self

    def save(self, path):
        p, _ = self.net.params()
        np.savez(path, params=p, n_knots=self.net.n_knots)

    def propose(self, L, J, beta_min, beta_max, n_temps=None, target_acceptance=None, max_temps=512):
        """(betas float64 [NT], eps float32 [NT - 1]) for one sample.  With
        n_temps None the net picks NT for target_acceptance per pair.  eps is
        capped at the invertibility bound of the sample."""
        return self.propose_many([(L, J, beta_min, beta_max)], n_temps, target_acceptance, max_temps)[0]

    def propose_many(self, samples, n_temps=None, target_acceptance=None, max_temps=512):
        """propose() for a list of (L, J, beta_min, beta_max) in one call."""
        x = np.stack([features(L, J, a, b) for (L, J, a, b) in samples])
        bmin = np.array([s[2] for s in samples], np.float64)
        bmax = np.array([s[3] for s in samples], np.float64)
        if n_temps is None:
            if target_acceptance is None:
                raise ValueError("give n_temps or target_acceptance")
            nt, sig = 0, float(sigma_of_acceptance(target_acceptance))
        else:
            nt, sig = n_temps, 0.0
        out = self.net.ladder(x, bmin, bmax, nt, KAPPA_MAX, sigma_target=sig, max_temps=max_temps)
        return [(b, np.minimum(e, eps_bound(L, J)).astype(np.float32))
                for (b, e), (L, J, _, _) in zip(out, samples)]

    def predicted_length(self, L, J, beta_min, beta_max):
        """Lambda = exp(z_{2P}): total sigma of an equal-acceptance ladder."""
        z = self.net.forward(features(L, J, beta_min, beta_max)[None])
        return float(np.exp(np.float64(z[0, -1])))

    def close(self):
        self.net.close()


def geometric_reference(L, J, beta_min, beta_max, n_temps, kappa):
    """The fallback: geometric ladder and one kappa for all pairs."""
    b = geometric(beta_min, beta_max, n_temps)
    return b, eps_from_kappa(b, np.full(n_temps - 1, kappa), eps_bound(L, J))


# ---------------------------------------------------------------- data set
def training_rows(seed_base=5000):
    """The training cases: lattice sizes TRAIN_L, inverse-temperature windows
    TRAIN_WINDOWS (three coupling samples each up to L = 16; at L = 24 and 32
    one sample of the paper's window and of [2, 8]), replica counts by
    default_n_temps."""
    rows = []
    for L in TRAIN_L:
        windows = TRAIN_WINDOWS if L <= 16 else ((2.0, 8.0), PAPER_WINDOW)
        n_seeds = 3 if L <= 16 else 1
        for w, (a, b) in enumerate(windows):
            for k in range(n_seeds):
                rows.append(Row(L, workloads.couplings(L, seed_base + 100 * L + 10 * w + k), a, b))
    return rows


def generate(path=TRAIN_FILE, n_cycles=2000, n_burn=1000, seed=0):
    """Run the kappa scans of training_rows() on the GPU and store features,
    targets and the measured acceptances (a few hundred KB)."""
    rows = training_rows()
    X, T, info = training_targets(rows, n_cycles=n_cycles, n_burn=n_burn, seed=seed)
    acc = np.concatenate([i["acc"] for i in info], axis=1)
    off = np.cumsum([0] + [r.n_temps - 1 for r in rows])
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.savez_compressed(path, X=X, T=T, L=np.array([r.L for r in rows]),
                        beta_min=np.array([r.beta_min for r in rows]),
                        beta_max=np.array([r.beta_max for r in rows]),
                        n_temps=np.array([r.n_temps for r in rows]), acc=acc, acc_offsets=off,
                        kappas=np.array(KAPPA_GRID), n_cycles=n_cycles, n_burn=n_burn)
    return X, T


def train(X, T, steps=4000, lr=2e-3, w_kappa=1.0, seed=1, stream=None):
    """Train a fresh net on the device; returns (LearnedLadder, losses)."""
    net = LearnedLadder(N_KNOTS, seed=seed, stream=stream)
    losses = net.train(X, T, steps=steps, lr=lr, w_kappa=w_kappa, record=True)
    return net, losses


def main(argv=None):
    ap = argparse.ArgumentParser(description="learned ladder: generate the training set / train the net")
    ap.add_argument("command", choices=["generate", "train"])
    ap.add_argument("--cycles", type=int, default=2000)
    ap.add_argument("--burn", type=int, default=1000)
    ap.add_argument("--steps", type=int, default=4000)
    a = ap.parse_args(argv)
    if a.command == "generate":
        X, T = generate(n_cycles=a.cycles, n_burn=a.burn)
        print(f"wrote {TRAIN_FILE}: {X.shape[0]} rows")
    else:
        d = np.load(TRAIN_FILE)
        net, losses = train(d["X"], d["T"], steps=a.steps)
        net.save(WEIGHTS_FILE)
        print(f"wrote {WEIGHTS_FILE}: loss {losses[0]:.4g} -> {losses[-1]:.4g}")


if __name__ == "__main__":
    main()
