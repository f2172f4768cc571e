"""Precision study at L = 32 (16 samples x 48 replicas x 2 copies, decimation
exchange): error of the float and the double engine against the FP64 oracle
per operation, and a paired long-run comparison of float against double.

Per operation (sampled replicas / chains of the full-size engine, one
operation from an identical state):
  heat-bath sweep, overrelaxation sweep  -> max |spin component| error
  energy                                  -> max relative error
  overlap chi                             -> max relative error
  decimation exchange                     -> decisions equal to the oracle's
Long run (paired: the float and double engines share couplings, initial
spins and Philox streams; per chain the difference of time averages, mean and
standard error over the 32 chains): energy per site at every beta, the
acceptance of every pair, chi at every beta.  The numbers are printed (run
with -s).
"""
import json
import os

import numpy as np
import pytest

import oracle as orc
from gpu_util import ambiguous_basis_sites, check_float_walk, exchange_walk, float_tolerances, site_colour
from paper_1006_4247_gb300 import pt
from paper_1006_4247_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NAME = "L32_R48_S16"
SAMPLED = [(2, 0, 5), (11, 1, 40)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1006_4247_gb300 import _build
    _build.build()


def _engine(precision, seed=3):
    w = W.WORKLOADS[NAME]()
    J = np.stack(w.couplings())
    B = np.stack(w.betas())
    eng = pt.Engine(w.L[0], J, B, n_copies=2, precision=precision, seed=seed)
    return w, eng, J.astype(np.float64), B


def _sweep_error(L, J, before, after, kind, beta, seed, sample, rep_id, step0, precision):
    col = site_colour(L)
    cur = before.copy()
    err = 0.0
    for colour in (0, 1):
        if kind == "hb":
            ref = orc.hb_halfsweep(L, J, cur, colour, beta, seed, sample, rep_id, step0 + colour)
            amb = ambiguous_basis_sites(L, J, cur, colour) if precision == "fp32" else np.zeros(L ** 3, bool)
        else:
            ref = orc.or_halfsweep(L, J, cur, colour)
            amb = np.zeros(L ** 3, bool)
        m = (col == colour) & ~amb
        err = max(err, float(np.abs(after[m] - ref[m]).max()))
        cur = cur.copy()
        cur[col == colour] = after[col == colour]
    return err


def test_per_operation_errors_against_oracle():
    report = {}
    for precision in ("fp32", "fp64"):
        w, eng, J, B = _engine(precision)
        L, NT = w.L[0], w.n_replicas[0]
        eng.sweep(1, 4)
        errs = {}
        for kind, (nh, no) in (("hb", (1, 0)), ("or", (0, 1))):
            before = {t: eng.get_spins(*t) for t in SAMPLED}
            step0 = eng.step
            eng.sweep(nh, no)
            errs[kind] = max(_sweep_error(L, J[s], before[(s, c, b)], eng.get_spins(s, c, b), kind, B[s, b], 3, s,
                                          c * NT + b, step0, precision) for (s, c, b) in SAMPLED)
        H = eng.energies()
        Q, chi = eng.overlap()
        e_rel, c_rel = 0.0, 0.0
        for (s, c, b) in SAMPLED:
            sp = eng.get_spins(s, c, b)
            Hr = orc.energy(L, J[s], sp)
            e_rel = max(e_rel, abs(H[s, c, b] - Hr) / abs(Hr))
            _, chir = orc.overlap(L, eng.get_spins(s, 0, b), eng.get_spins(s, 1, b))
            c_rel = max(c_rel, abs(chi[s, b] - chir) / chir)
        errs["energy_rel"] = e_rel
        errs["chi_rel"] = c_rel
        # one decimation exchange of a sampled chain against the oracle
        s, c = SAMPLED[0][0], SAMPLED[0][1]
        st = np.stack([eng.get_spins(s, c, b) for b in range(NT)])
        prop, acc, rt, perm = eng.stats()
        ch = orc.Chain(L, J[s], B[s], st, copy=c, sample=s, seed=3)
        ch.label[:] = perm[s, c]
        acc0 = acc[s, c].copy()
        step = eng.step
        eng.exchange("decimation")
        ch.exchange(1, step)
        prop, acc, rt, perm = eng.stats()
        errs["decisions_equal"] = bool((perm[s, c] == ch.label).all() and ((acc[s, c] - acc0) == ch.acc).all())
        report[precision] = errs
        eng.close()
    print("\nprecision study, per operation:", json.dumps(report))
    assert report["fp32"]["hb"] <= 1e-5 and report["fp32"]["or"] <= 1e-5
    assert report["fp64"]["hb"] <= 1e-12 and report["fp64"]["or"] <= 1e-12
    assert report["fp32"]["energy_rel"] <= 2e-5 and report["fp64"]["energy_rel"] <= 1e-11
    assert report["fp32"]["chi_rel"] <= 1e-4 and report["fp64"]["chi_rel"] <= 1e-10
    assert report["fp64"]["decisions_equal"]


def test_paired_long_run_float_vs_double():
    cycles, burn = 60, 20
    res = {}
    for precision in ("fp32", "fp64"):
        w, eng, J, B = _engine(precision, seed=11)
        S, NT, L = w.n_samples, w.n_replicas[0], w.L[0]
        e = np.zeros((cycles, S, 2, NT))
        x = np.zeros((cycles, S, NT))
        for k in range(cycles):
            eng.sweep(w.n_hb, w.n_or)
            eng.exchange(w.exchange)
            h, q, c = eng.measure()
            e[k] = h.reshape(S, 2, NT) / L ** 3
            x[k] = c.reshape(S, NT)
        prop, acc, rt, perm = eng.stats()
        res[precision] = (e[burn:].mean(0).reshape(S * 2, NT), x[burn:].mean(0),
                          (acc / np.maximum(prop, 1)).reshape(S * 2, NT - 1))
        eng.close()
    out = {}
    zs = []
    for k, name in enumerate(("energy_per_site", "chi", "acceptance")):
        d = res["fp32"][k] - res["fp64"][k]
        m, se = d.mean(0), d.std(0, ddof=1) / np.sqrt(d.shape[0])
        z = np.abs(m) / np.maximum(se, 1e-300)
        zs.append(z)
        out[name] = {"max_abs_mean_diff": float(np.abs(m).max()), "max_z": float(z.max())}
    print("\nprecision study, paired float - double:", json.dumps(out))
    z = np.concatenate(zs)
    assert (z < 2.0).mean() >= 0.85 and z.max() < 5.0


def test_coolheat_errors_against_oracle():
    """Cooling/heating at L = 16 (64 samples x 24 replicas x 2 copies, the
    configuration-2 batch, staged exchange kernels; cooling parameter
    kappa = 0.1, eps_i = kappa ln(beta_{i+1}/beta_i), so that about a third of
    the pairs accept): one tempering update of sampled chains from an
    identical state, float and double engines, against the oracle walk
    (which follows the engine's decisions).  Reported per precision: the
    largest error of a sweep's ln det J_C, of a pair's ln A, of a transformed
    spin component, and the pairs decided differently (round-off ties)."""
    name = "L16_R24_S64"
    chains = [(4, 0), (21, 1), (50, 0), (63, 1)]
    report = {}
    for precision in ("fp32", "fp64"):
        w = W.WORKLOADS[name]()
        J = np.stack(w.couplings())
        B = np.stack(w.betas())
        eng = pt.Engine(w.L[0], J, B, n_copies=2, precision=precision, seed=5)
        L, NT, S = w.L[0], w.n_replicas[0], w.n_samples
        eps = np.stack([(0.1 * np.log(B[s, 1:] / B[s, :-1])).astype(np.float32) for s in range(S)])
        eng.set_params(eps=eps)
        Jd = J.astype(np.float64)
        for _ in range(2):
            eng.sweep(w.n_hb, w.n_or)
            eng.exchange("coolheat")
        eng.sweep(w.n_hb, w.n_or)
        H0 = eng.energies()
        step = eng.step
        start = {(s, c): np.stack([eng.get_spins(s, c, b) for b in range(NT)]) for (s, c) in chains}
        perm0 = eng.stats()[3]
        eng.exchange("coolheat")
        perm1 = eng.stats()[3]
        lnA, lnJ = eng.exchange_log()
        errors = {}
        n_acc = 0
        for (s, c) in chains:
            recs, sp, Hw, permw = exchange_walk("coolheat", L, Jd[s], B[s], start[(s, c)], H0[s, c], 5, s, c, step,
                                                eps=eps[s], follow_lnA=lnA[s, c])
            float_tolerances(recs, "coolheat", B[s], L ** 3)
            check_float_walk(errors, name, lnA[s, c], lnJ[s, c], recs, L ** 3)
            assert (perm1[s, c] == perm0[s, c][permw]).all(), (precision, s, c)
            d = max(float(np.abs(eng.get_spins(s, c, b) - sp[b]).max()) for b in range(NT))
            errors[name]["spin"] = max(errors[name]["spin"], d)
            n_acc += sum(bool(r["accepted"]) for r in recs)
        errors[name]["accepted_pairs"] = int(n_acc)
        report[precision] = errors[name]
        eng.close()
    print("\nprecision study, cooling/heating:", json.dumps(report))
    assert report["fp64"]["ties"] == 0
    assert report["fp64"]["lnA"] <= 1e-8 and report["fp64"]["lnJ"] <= 1e-9 and report["fp64"]["spin"] <= 1e-12
    assert report["fp32"]["spin"] <= 1e-5 and report["fp32"]["lnJ"] <= 16 ** 3 * 1e-6
    assert report["fp32"]["accepted_pairs"] > 0
