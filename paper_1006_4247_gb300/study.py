"""The paper's measurement protocol (section IV) on synthetic coupling sets.

For one lattice size: ``n_sets`` Gaussian coupling sets, the geometric ladder
of the paper (T from 0.12 to 0.19, N_T replicas), two copies per set, update
cycles of 1 heat-bath + 5L/4 overrelaxation sweeps and one tempering update,
run with each exchange method on the same sets.  Reported per method:

* the acceptance of every pair (Table I gives the first and last pair);
* the round-trip time t_R: sweeps of the run divided by the round trips of
  all 2 N_T configurations of a set (section IV.B);
* the integrated autocorrelation time of the overlap susceptibility at the
  lowest temperature, tau_int(chi) in sweeps, by automatic windowing (the
  smallest window W with W >= c tau(W), c = 4; Sokal).

The paper's coupling sets are not available, so the absolute values are not
comparable with its tables; the ratios between methods are the result.  All
work runs in the engine (C ABI); this module only drives it and reduces the
measurements on the host.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import ladder
from . import pt
from . import workloads

T_MIN, T_MAX = 0.12, 0.19


def paper_ladder(n_temps: int) -> np.ndarray:
    """beta_i of the paper's geometric temperature ladder, ascending."""
    return ladder.geometric(1.0 / T_MAX, 1.0 / T_MIN, n_temps)


def tau_int(x: np.ndarray, c: float = 4.0) -> float:
    """Integrated autocorrelation time (in samples) of a series by automatic
    windowing: tau(W) = 1/2 + sum_{t=1}^{W} rho(t), the first W >= c tau(W)."""
    x = np.asarray(x, np.float64)
    n = x.size
    if n < 8:
        return float("nan")
    y = x - x.mean()
    f = np.fft.rfft(y, 2 * n)
    acf = np.fft.irfft(f * np.conj(f))[:n]
    if acf[0] <= 0:
        return float("nan")
    rho = acf / acf[0]
    tau = 0.5
    for W in range(1, n):
        tau += rho[W]
        if W >= c * tau:
            return float(tau)
    return float(tau)


def run_method(L, couplings, betas, mode, eps, cycles, burn, seed=0):
    """One engine run of all sets with one exchange method; betas [NT] or per
    set [S, NT], eps [NT-1] or [S, NT-1] (or None).  Returns the acceptance
    per set and pair [S, NT-1], round trips per set [S] and the chi series at
    the lowest temperature [cycles, S] (after the burn-in)."""
    import torch
    S = len(couplings)
    B = np.asarray(betas, np.float64)
    NT = B.shape[-1]
    n_or = max(1, (5 * L) // 4)
    stream = torch.cuda.Stream()
    eng = pt.Engine(L, np.stack(couplings), np.broadcast_to(B, (S, NT)).copy(), n_copies=2, seed=seed,
                    stream=stream.cuda_stream)
    try:
        if eps is not None:
            eng.set_params(None, np.broadcast_to(eps, (S, NT - 1)).astype(np.float32).copy())
        eng.autotune(1, n_or)
        eng.cycles(burn, 1, n_or, mode)
        p0, a0, r0, _ = eng.stats()
        chi = torch.empty((cycles, S * NT), dtype=torch.float64, device="cuda")
        for k in range(cycles):
            eng.cycles(1, 1, n_or, mode)
            eng.measure_device(d_chi=chi[k])
        torch.cuda.synchronize()
        p1, a1, r1, _ = eng.stats()
    finally:
        eng.close()
    acc = (a1 - a0).sum(1) / np.maximum((p1 - p0).sum(1), 1)  # pooled over the copies
    rt = (r1 - r0).sum(1)
    chi_min_T = chi.view(cycles, S, NT)[:, :, NT - 1].cpu().numpy()
    return acc, rt, chi_min_T


def protocol(L, n_temps, n_sets=10, cycles=20000, burn=5000, kappa=0.1, seed0=8000,
             methods=("plain", "decimation", "coolheat")):
    """The protocol for one L; returns a JSON-ready summary."""
    J = [workloads.couplings(L, seed0 + 97 * L + k) for k in range(n_sets)]
    b = paper_ladder(n_temps)
    spc = 1 + max(1, (5 * L) // 4)  # sweeps per cycle
    out = {"L": L, "n_temps": n_temps, "n_sets": n_sets, "cycles": cycles, "burn": burn,
           "sweeps_per_cycle": spc, "kappa": kappa, "methods": {}}
    for m in methods:
        eps = None
        if m == "coolheat":
            bound = min(ladder.eps_bound(L, j) for j in J)
            eps = ladder.eps_from_kappa(b, np.full(n_temps - 1, kappa), bound)
        acc, rt, chi = run_method(L, J, b, m, eps, cycles, burn, seed=11)
        tR = cycles * spc / np.maximum(rt, 1)
        tau = np.array([tau_int(chi[:, s]) * spc for s in range(n_sets)])
        out["methods"][m] = {
            "acc_first_pair": [float(acc[:, 0].min()), float(acc[:, 0].max())],
            "acc_last_pair": [float(acc[:, -1].min()), float(acc[:, -1].max())],
            "acc_mean": float(acc.mean()),
            "acc_profile": acc.mean(0).round(4).tolist(),
            "t_R": [float(tR.min()), float(tR.max())],
            "t_R_per_set": tR.round(1).tolist(),
            "round_trips_per_set": rt.tolist(),
            "tau_int_chi": [float(np.nanmin(tau)), float(np.nanmax(tau))],
            "tau_int_chi_per_set": np.round(tau, 1).tolist(),
        }
    ms = out["methods"]
    if "plain" in ms:
        # speed-ups over the standard method, averaged over the sets (Table II)
        tp = np.array(ms["plain"]["t_R_per_set"])
        taup = np.array(ms["plain"]["tau_int_chi_per_set"])
        for m in ms:
            if m != "plain":
                ms[m]["t_R_speedup_mean"] = float(np.mean(tp / np.array(ms[m]["t_R_per_set"])))
                r = taup / np.array(ms[m]["tau_int_chi_per_set"])
                ms[m]["tau_speedup_mean"] = float(np.nanmean(r))
                ms[m]["tau_speedup_median"] = float(np.nanmedian(r))  # robust to sets not yet equilibrated
                ms[m]["acc_ratio"] = ms[m]["acc_mean"] / ms["plain"]["acc_mean"]
    return out


def replicas(L, n_temps_list, reference_nt, n_sets=10, cycles=20000, burn=5000, kappa=0.1, seed0=8000,
             plain_all=True):
    """Round-trip time against the number of replicas (the
    paper's reduced-N_T test generalised) for: the standard swap, decimation
    and cooling/heating on the geometric ladder (one kappa), and
    cooling/heating on the ladders and epsilons the learned network proposes
    for each set.  Returns t_R per (arm, N_T) (mean over sets, sweeps) and,
    per arm, the smallest N_T whose t_R is not above the standard method's at
    reference_nt.  plain_all=False runs the standard swap at reference_nt
    only (all the comparison needs)."""
    J = [workloads.couplings(L, seed0 + 97 * L + k) for k in range(n_sets)]
    spc = 1 + max(1, (5 * L) // 4)
    net = ladder.LearnedLadder.load()
    arms = ("plain", "decimation", "coolheat", "coolheat_learned")
    out = {"L": L, "reference_nt": reference_nt, "n_sets": n_sets, "cycles": cycles, "burn": burn,
           "sweeps_per_cycle": spc, "t_R": {a: {} for a in arms}, "acc_min": {a: {} for a in arms},
           "t_R_se": {a: {} for a in arms}, "tau_int_median": {a: {} for a in arms}}
    try:
        for nt in sorted(set(list(n_temps_list) + [reference_nt])):
            b = paper_ladder(nt)
            for arm in arms:
                if arm == "plain" and nt != reference_nt and (not plain_all or nt < min(n_temps_list)):
                    continue
                mode = "coolheat" if arm.startswith("coolheat") else arm
                eps = None
                betas = b
                if arm == "coolheat":
                    bound = min(ladder.eps_bound(L, j) for j in J)
                    eps = ladder.eps_from_kappa(b, np.full(nt - 1, kappa), bound)
                elif arm == "coolheat_learned":
                    prop = net.propose_many([(L, j, 1 / T_MAX, 1 / T_MIN) for j in J], n_temps=nt)
                    betas = np.stack([p[0] for p in prop])
                    eps = np.stack([p[1] for p in prop])
                acc, rt, chi = run_method(L, J, betas, mode, eps, cycles, burn, seed=13)
                tR = cycles * spc / np.maximum(rt, 1)
                # sweeps to decorrelate chi at the lowest temperature (c = 4), median over the sets
                out["tau_int_median"][arm][nt] = float(np.median([tau_int(chi[:, k]) * spc for k in range(n_sets)]))
                out["t_R"][arm][nt] = float(tR.mean())
                out["t_R_se"][arm][nt] = float(tR.std(ddof=1) / math.sqrt(n_sets))
                out["acc_min"][arm][nt] = float(acc.min(1).mean())
    finally:
        net.close()
    ref = out["t_R"]["plain"][reference_nt]
    out["replicas_needed"] = {a: min([nt for nt, t in out["t_R"][a].items() if t <= ref], default=None) for a in arms}
    return out


def equilibration(L=16, n_temps=15, n_runs=2000, cycles=1000, kappa=0.1, seed=8500,
                  methods=("plain", "decimation", "coolheat")):
    """Equilibration from the ordered start (section IV.C, Fig. 1):
    n_runs independent runs (independent random numbers) on one coupling set,
    every spin (1, 0, 0) at the start, all runs in one batched engine; the
    mean and standard error over runs of chi at the lowest temperature after
    every cycle.  Returns the curve at a few cycle counts per method and the
    first cycle where the mean comes within 5% of its value over the last
    tenth of the run."""
    import torch
    J = workloads.couplings(L, seed)
    b = paper_ladder(n_temps)
    n_or = max(1, (5 * L) // 4)
    marks = [m for m in (1, 3, 10, 30, 100, 300, 1000, 3000) if m <= cycles]
    out = {"L": L, "n_temps": n_temps, "runs": n_runs, "cycles": cycles, "marks": marks, "methods": {}}
    for m in methods:
        eps = None
        if m == "coolheat":
            eps = ladder.eps_from_kappa(b, np.full(n_temps - 1, kappa), ladder.eps_bound(L, J))
        stream = torch.cuda.Stream()
        eng = pt.Engine(L, np.broadcast_to(J, (n_runs,) + J.shape).copy(), np.broadcast_to(b, (n_runs, n_temps)).copy(),
                        n_copies=2, seed=seed + 1, start="ordered", stream=stream.cuda_stream)
        try:
            if eps is not None:
                eng.set_params(None, np.broadcast_to(eps, (n_runs, n_temps - 1)).astype(np.float32).copy())
            chi = torch.empty((cycles, n_runs * n_temps), dtype=torch.float64, device="cuda")
            for k in range(cycles):
                eng.cycles(1, 1, n_or, m)
                eng.measure_device(d_chi=chi[k])
            torch.cuda.synchronize()
        finally:
            eng.close()
        c = chi.view(cycles, n_runs, n_temps)[:, :, n_temps - 1]
        mean = c.mean(1).cpu().numpy()
        se = (c.std(1) / math.sqrt(n_runs)).cpu().numpy()
        plateau = float(mean[-max(1, cycles // 10):].mean())
        close = np.nonzero(np.abs(mean - plateau) <= 0.05 * abs(plateau))[0]
        out["methods"][m] = {"chi": [float(mean[t - 1]) for t in marks], "se": [float(se[t - 1]) for t in marks],
                             "plateau": plateau, "cycles_to_5pct": int(close[0]) + 1 if close.size else None,
                             "curve_every_10": mean[9::10].round(3).tolist()}
    if "plain" in out["methods"]:
        # cycles each method needs to reach the standard method's chi after 30%, 100% of the run
        ref = out["methods"]["plain"]["curve_every_10"]
        for m, v in out["methods"].items():
            cur = np.array(v["curve_every_10"])
            v["cycles_to_reach_standard"] = {}
            for frac in (0.3, 1.0):
                target = ref[max(0, int(frac * len(ref)) - 1)]
                hit = np.nonzero(cur >= target)[0]
                v["cycles_to_reach_standard"][str(frac)] = int(10 * (hit[0] + 1)) if hit.size else None
    return out


def learned_large(L=48, n_samples=32, n_run=8, cycles=300, burn=200, kappa=0.1, seed0=400):
    """The learned ladder on a size far outside its training range (L = 48,
    coupling seeds 400 + k): proposals for n_samples sets, and a short
    acceptance comparison on n_run of them against the geometric ladder with
    the paper's replica rule and one kappa.  The network picks N_T for the
    geometric arm's measured worst-pair acceptance.  Round trips are not
    measured (t_R at L = 48 is far beyond a short run)."""
    J = [workloads.couplings(L, seed0 + k) for k in range(n_samples)]
    bmin, bmax = 1 / T_MAX, 1 / T_MIN
    nt_geo = ladder.default_n_temps(L, bmin, bmax)
    geo = paper_ladder(nt_geo)
    bound = min(ladder.eps_bound(L, j) for j in J[:n_run])
    eps_geo = ladder.eps_from_kappa(geo, np.full(nt_geo - 1, kappa), bound)
    acc_g, _, _ = run_method(L, J[:n_run], geo, "coolheat", eps_geo, cycles, burn, seed=17)
    target = float(acc_g.min(1).mean())
    net = ladder.LearnedLadder.load()
    try:
        lam = [net.predicted_length(L, j, bmin, bmax) for j in J]
        auto = net.propose_many([(L, j, bmin, bmax) for j in J], target_acceptance=target)
    finally:
        net.close()
    nts = [len(b) for b, _ in auto]
    nt_l = max(nts[:n_run])  # one engine needs one N_T: the largest the net asks for among the runs
    net = ladder.LearnedLadder.load()
    try:
        run = net.propose_many([(L, j, bmin, bmax) for j in J[:n_run]], n_temps=nt_l)
    finally:
        net.close()
    acc_l, _, _ = run_method(L, J[:n_run], np.stack([b for b, _ in run]), "coolheat", np.stack([e for _, e in run]),
                             cycles, burn, seed=17)
    kap = [float(np.mean(e / np.diff(np.log(b)))) for b, e in run]
    return {"L": L, "samples": n_samples, "run_samples": n_run, "cycles": cycles, "burn": burn,
            "geometric": {"n_temps": nt_geo, "kappa": kappa, "acc_min": target, "acc_mean": float(acc_g.mean()),
                          "acc_profile": acc_g.mean(0).round(4).tolist()},
            "learned": {"n_temps_proposed": nts, "n_temps_run": nt_l, "predicted_Lambda": [round(x, 2) for x in lam],
                        "kappa_mean": float(np.mean(kap)), "acc_min": float(acc_l.min(1).mean()),
                        "acc_mean": float(acc_l.mean()), "acc_profile": acc_l.mean(0).round(4).tolist()}}


def learned_large_roundtrip(L=48, n_run=8, cycles=3000, burn=1500, kappa=0.1, seed0=400, reduce=0.85):
    """Round trips at a size outside the network's training range (L = 48,
    coupling seeds 400 + k, the first n_run sets): the geometric ladder with
    one kappa and the learned ladder with its per-pair epsilon, each at the
    paper's replica rule N_T and at round(reduce * N_T) replicas, after a
    burn-in from a random start.  Reported per arm: t_R (sweeps of the
    measured cycles over the round trips of all 2 N_T configurations, mean
    and standard error over the sets), the median tau_int(chi) at the lowest
    temperature in sweeps, and the acceptance (worst pair, mean)."""
    J = [workloads.couplings(L, seed0 + k) for k in range(n_run)]
    bmin, bmax = 1 / T_MAX, 1 / T_MIN
    spc = 1 + max(1, (5 * L) // 4)
    nt_full = ladder.default_n_temps(L, bmin, bmax)
    nt_red = int(round(reduce * nt_full))
    bound = min(ladder.eps_bound(L, j) for j in J)
    out = {"L": L, "sets": n_run, "cycles": cycles, "burn": burn, "sweeps_per_cycle": spc, "kappa": kappa,
           "n_temps": [nt_full, nt_red], "arms": {}}
    for nt in (nt_full, nt_red):
        geo = paper_ladder(nt)
        net = ladder.LearnedLadder.load()
        try:
            prop = net.propose_many([(L, j, bmin, bmax) for j in J], n_temps=nt)
        finally:
            net.close()
        arms = {"geometric": (geo, ladder.eps_from_kappa(geo, np.full(nt - 1, kappa), bound)),
                "learned": (np.stack([b for b, _ in prop]), np.stack([e for _, e in prop]))}
        for name, (betas, eps) in arms.items():
            acc, rt, chi = run_method(L, J, betas, "coolheat", eps, cycles, burn, seed=19)
            tR = cycles * spc / np.maximum(rt, 1)
            tau = [tau_int(chi[:, k]) * spc for k in range(n_run)]
            out["arms"][f"{name}_{nt}"] = {
                "n_temps": nt, "t_R": float(tR.mean()), "t_R_se": float(tR.std(ddof=1) / math.sqrt(n_run)),
                "round_trips_per_set": rt.tolist(), "tau_int_median": float(np.nanmedian(tau)),
                "acc_min": float(acc.min(1).mean()), "acc_mean": float(acc.mean()),
                "acc_profile": acc.mean(0).round(4).tolist()}
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description="the paper's protocol on synthetic coupling sets")
    ap.add_argument("--L", type=int, default=16)
    ap.add_argument("--n-temps", type=int, default=0, help="0: the paper's N_T (15, 27, 43 at L = 16, 24, 32)")
    ap.add_argument("--sets", type=int, default=10)
    ap.add_argument("--cycles", type=int, default=20000)
    ap.add_argument("--burn", type=int, default=5000)
    ap.add_argument("--kappa", type=float, default=0.1)
    ap.add_argument("--methods", default="plain,decimation,coolheat")
    ap.add_argument("--replicas", default="", help="comma-separated N_T list: run the replica-count study")
    ap.add_argument("--plain-reference-only", action="store_true",
                    help="replica study: the standard swap at the paper's N_T only")
    ap.add_argument("--equilibration", type=int, default=0, help="runs of the equilibration study (0: off)")
    ap.add_argument("--learned-large", action="store_true", help="learned ladder at L (e.g. 48) vs geometric")
    ap.add_argument("--learned-large-rt", action="store_true",
                    help="round trips of the learned and the geometric ladder at L (e.g. 48), full and reduced N_T")
    ap.add_argument("--run-sets", type=int, default=8, help="--learned-large-rt: coupling sets run")
    ap.add_argument("--log", default="", help="also append the result as a JSON-lines run record to this file")
    a = ap.parse_args(argv)
    nt = a.n_temps or {16: 15, 24: 27, 32: 43}.get(a.L, ladder.default_n_temps(a.L, 1 / T_MAX, 1 / T_MIN))
    if a.learned_large_rt:
        kind, out = "learned_large_rt", learned_large_roundtrip(a.L, a.run_sets, a.cycles, a.burn, a.kappa)
    elif a.learned_large:
        kind, out = "learned_large", learned_large(a.L, cycles=a.cycles, burn=a.burn)
    elif a.equilibration:
        kind, out = "equilibration", equilibration(a.L, nt, a.equilibration, a.cycles, a.kappa)
    elif a.replicas:
        nts = [int(v) for v in a.replicas.split(",")]
        kind, out = "replicas", replicas(a.L, nts, nt, a.sets, a.cycles, a.burn, a.kappa,
                                         plain_all=not a.plain_reference_only)
    else:
        kind, out = "protocol", protocol(a.L, nt, a.sets, a.cycles, a.burn, a.kappa,
                                         methods=tuple(a.methods.split(",")))
    print(json.dumps(out))
    if a.log:
        from . import runlog
        cfg = {k: v for k, v in vars(a).items() if k != "log"}
        cfg["n_temps"] = nt
        runlog.record(a.log, "study_" + kind, cfg, out)


if __name__ == "__main__":
    main()
