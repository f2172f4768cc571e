#!/usr/bin/env python3
"""Throughput of the parallel-tempering hot path on GB300.

One step = one update cycle of every replica of every chain of the workload:
1 heat-bath sweep + 5L/4 overrelaxation sweeps (section IV of Hasenbusch &
Schaefer), the energy reduction, one tempering update (the exchange mode of
the workload) and the overlap reduction.  The metric is site updates per
nanosecond (each sweep updates every site of every replica once), reported
beside the HBM roofline of the dominant kernel (the overrelaxation half
sweep).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                  [--exchange plain|decimation|coolheat] [--impl ours|reference]

Under torchrun every rank runs its own disorder samples (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1006_4247_gb300 import sharding  # noqa: E402
from paper_1006_4247_gb300 import workloads as W  # noqa: E402

HBM_FALLBACK_GBS = 6800.0
L2_BYTES = 129e6


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--workload", default="L32_R48_S16",
                   choices=["L4_R8_S1", "L16_R24_S64", "L32_R48_S16", "uneven_S256"])
    p.add_argument("--exchange", default=None)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    p.add_argument("--policy", default="auto", choices=["auto", "streaming", "resident"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--log", default="", help="also append the line as a JSON-lines run record to this file")
    p.add_argument("--no-cpu", action="store_true")
    return p.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return HBM_FALLBACK_GBS, "fallback"


KERNEL_SOURCES = {
    "k_sweep": ("sweep.cu", "pt_device.cuh", "pt_types.h", "kernels.h"),
    "k_resident": ("resident.cu", "pt_device.cuh", "tma.cuh", "pt_types.h", "kernels.h"),
}


def kernel_source_hash(kernel):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1006_4247_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, workload, precision):
    """DRAM bytes (read + write) per launch of `kernel` from the committed ncu
    summary, if it was captured on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    e = d.get(f"{kernel}:{workload}:{precision}")
    if not e or e.get("source_hash") != kernel_source_hash(kernel):
        return None
    return float(e["dram_bytes_per_launch"])


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def workload_of(args, rank):
    if args.workload == "uneven_S256":
        w = W.uneven_batch()
        w.j_seed0 = sharding.coupling_seed0(w.j_seed0, rank)
        return w
    w = W.WORKLOADS[args.workload]()
    if args.exchange:
        w.exchange = args.exchange
    w.j_seed0 = sharding.coupling_seed0(w.j_seed0, rank)
    return w


def n_or_of(w):
    """Overrelaxation sweeps per sample: the workload's count, or 5L/4 per
    sample (section IV) for a batch of uneven L."""
    if "n_or_per_L" in w.extra:
        return [w.extra["n_or_per_L"][L] for L in w.L]
    return [w.n_or] * w.n_samples


def updates_per_step(w):
    return sum(w.n_copies * nt * L ** 3 * (w.n_hb + no) for L, nt, no in zip(w.L, w.n_replicas, n_or_of(w)))


def eps_array(w):
    return np.concatenate([np.full(nt - 1, w.eps, np.float32) for nt in w.n_replicas])


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and --impl reference)
# ---------------------------------------------------------------------------
def oracle_cycle_rate(w, budget_s=12.0, max_cycles=None):
    """Site updates/ns of the oracle on one sample of the workload, single
    thread, as it stands."""
    import oracle
    oracle.build()
    L, NT = w.L[0], w.n_replicas[0]
    J = W.couplings(L, w.j_seed0).astype(np.float64)
    B = W.linear_betas(NT, w.beta_min, w.beta_max)
    run = oracle.Run(L, J, B, n_copies=w.n_copies, seed=1, eps=w.eps)
    mode = {"plain": 0, "decimation": 1, "coolheat": 2}[w.exchange]
    nor0 = n_or_of(w)[0]  # the sample's own count (5L/4 in an uneven batch)
    per_cycle = w.n_copies * NT * L ** 3 * (w.n_hb + nor0)
    t0 = time.perf_counter()
    n = 0
    while True:
        run.cycles(1, w.n_hb, nor0, mode, record=False)
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s or (max_cycles and n >= max_cycles):
            break
    return per_cycle * n / (el * 1e9), n, el


def _oracle_worker(job):
    """One host process of the all-cores oracle leg: sample k of the workload
    (its own couplings), cycles for `budget_s` seconds; returns site updates."""
    (L, NT, j_seed, beta_min, beta_max, n_copies, eps, exchange, n_hb, n_or), k, budget_s = job
    import oracle
    J = W.couplings(L, j_seed + k).astype(np.float64)
    B = W.linear_betas(NT, beta_min, beta_max)
    run = oracle.Run(L, J, B, n_copies=n_copies, seed=1 + k, eps=eps)
    mode = {"plain": 0, "decimation": 1, "coolheat": 2}[exchange]
    per_cycle = n_copies * NT * L ** 3 * (n_hb + n_or)
    t0 = time.perf_counter()
    n = 0
    while time.perf_counter() - t0 < budget_s:
        run.cycles(1, n_hb, n_or, mode, record=False)
        n += 1
    return per_cycle * n


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_rate_all_cores(w, budget_s=12.0):
    """The same oracle, unchanged, run as one independent process per host
    core, each on its own sample of the workload (samples are independent
    chains): total site updates/ns over the wall time of the pool."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    n = host_cores()
    ctx = mp.get_context("spawn")
    spec = (w.L[0], w.n_replicas[0], w.j_seed0, w.beta_min, w.beta_max, w.n_copies, w.eps, w.exchange,
            w.n_hb, n_or_of(w)[0])  # the sample the single-thread leg times, other couplings per process
    with ctx.Pool(n) as pool:
        pool.map(_oracle_worker, [(spec, k, 0.2) for k in range(n)])  # interpreters started and warm
        t0 = time.perf_counter()
        ups = pool.map(_oracle_worker, [(spec, k, budget_s) for k in range(n)])
        el = time.perf_counter() - t0
    return sum(ups) / (el * 1e9), n, el


def reference_arm(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    w = workload_of(args, 0)
    import oracle
    oracle.build()
    L, NT = w.L[0], w.n_replicas[0]
    J = W.couplings(L, w.j_seed0).astype(np.float64)
    B = W.linear_betas(NT, w.beta_min, w.beta_max)
    mode = {"plain": 0, "decimation": 1, "coolheat": 2}[w.exchange]
    nor0 = n_or_of(w)[0]
    # one step = one cycle of one sample; where that is more than about 5 s of
    # single-thread work (L = 32: 1.3e8 site updates) only its first copy's
    # chain is run, so that the whole run stays within a few minutes
    copies = w.n_copies if w.n_copies * NT * L ** 3 * (w.n_hb + nor0) <= 8e7 else 1
    run = oracle.Run(L, J, B, n_copies=copies, seed=1, eps=w.eps)
    for _ in range(args.warmup):
        run.cycles(1, w.n_hb, nor0, mode, record=False)
    per_step = copies * NT * L ** 3 * (w.n_hb + nor0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run.cycles(1, w.n_hb, nor0, mode, record=True)
    el = time.perf_counter() - t0
    v = per_step * args.steps / (el * 1e9)
    sample = (f"one sample (L={L}, {NT} replicas x {copies} of its {w.n_copies} copies) of {w.name}, "
              "one cycle per step")
    line = {
        "metric": "site_updates_per_ns", "value": v, "unit": "updates/ns", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": w.name, "L": L, "replicas": NT, "copies": copies,
                   "samples": 1, "n_hb": w.n_hb, "n_or": nor0, "exchange": w.exchange},
        "cpu_baseline": {"value": v, "unit": "updates/ns", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "updates/ns", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    if args.log:
        from paper_1006_4247_gb300 import runlog
        runlog.record(args.log, "bench_reference", line["config"], {k: v for k, v in line.items() if k != "config"})


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def ours(args):
    import torch
    from paper_1006_4247_gb300 import _build, pt

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    _build.build()
    w = workload_of(args, rank)
    stream = torch.cuda.Stream()  # the engine's own stream (graphs need one)
    uniform = len(set(w.L)) == 1 and len(set(w.n_replicas)) == 1
    if uniform:
        eng = pt.Engine(w.L[0], np.stack(w.couplings()), np.stack(w.betas()), n_copies=w.n_copies,
                        precision=args.precision, seed=sharding.engine_seed(rank), stream=stream.cuda_stream)
    else:
        eng = pt.Engine(list(w.L), w.couplings(), w.betas(), n_copies=w.n_copies, precision=args.precision,
                        seed=sharding.engine_seed(rank), stream=stream.cuda_stream)
    eps = eps_array(w)
    eng.set_params(eps=eps)
    mode = w.exchange
    nor = n_or_of(w)
    nor_samples = None if len(set(nor)) == 1 else nor
    tune = None
    if args.policy == "auto" and not args.no_autotune:
        tune = eng.autotune(w.n_hb, max(nor))  # the block as the cycle runs it
    else:
        eng.set_policy(args.policy)

    def step(graph=True):
        if graph:
            eng.cycles(1, w.n_hb, nor[0], mode, measure=True, n_or_samples=nor_samples)
        else:
            if nor_samples is None:
                eng.sweep(w.n_hb, nor[0])
            else:
                eng.sweep_samples(w.n_hb, nor_samples)
            eng.exchange(mode)
            eng.measure_device()

    def barrier():
        sharding.barrier(torch.cuda.synchronize)

    def timed(nsteps, profile):
        eng.profile(profile)
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(nsteps):
            step(graph=not profile)
        ev1.record(stream)
        barrier()
        t = ev0.elapsed_time(ev1)
        pm, ln = eng.profile_read()
        eng.profile(False)
        return t, pm, ln

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    # the shared-memory data path's measured rate: the resident blocks' roofline
    smem_Bps, smem_bpc, smem_mhz = pt.pt_smem_bandwidth(stream.cuda_stream)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ms, _, launches = timed(args.steps, profile=False)
    clk = clocks.stop()
    # a shorter profiled pass (events around every launch) for per-kernel times
    _, prof_ms, prof_launches = timed(max(2, args.steps // 2), profile=True)
    ms = sharding.max_over_ranks(ms, device="cuda")
    ups = updates_per_step(w)
    value = sharding.weak_throughput(ups, args.steps, world, ms, 1e6)
    n_prof_steps = max(2, args.steps // 2)

    bpe = 4 if args.precision == "fp32" else 8
    peak, peak_src = load_peaks()
    resident = [bool(tune is not None and tune[0][s] >= 10) for s in range(w.n_samples)] if tune is not None \
        else [args.policy == "resident"] * w.n_samples
    if tune is None and args.policy == "auto":
        resident = [False] * w.n_samples

    def or_roofline(pm, ln, res_flags, steps):
        """HBM roofline of the streaming overrelaxation half sweeps: 36 B per
        update in float (read own + write own + read the other colour) plus
        each sample's couplings once per half sweep."""
        alg = 0
        for s, (L, nt, no) in enumerate(zip(w.L, w.n_replicas, nor)):
            if res_flags[s]:
                continue
            N = L ** 3
            alg += (w.n_copies * nt * (N // 2) * 9 * bpe + 3 * N * 4) * 2 * no
        alg *= steps
        if pm["or"] <= 0 or alg == 0:  # no event time (e.g. launches serialised by a profiler)
            return None
        ach = alg / (pm["or"] / 1e3) / 1e9
        n_launch = max(ln["or"], 1)
        kern = "k_sweep"
        wl = w.name if uniform else None
        return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": ncu_traffic(kern, wl, args.precision) if wl else None,
                "kernel": "k_sweep<OR> (streaming half sweep)", "peak_source": peak_src,
                "alg_bytes_per_launch": alg / n_launch, "avg_launch_us": pm["or"] / n_launch * 1e3}

    def resident_roofline(pm, ln, res_flags, steps):
        """The resident block reads and writes each replica once per cycle
        through HBM and runs every half sweep out of shared memory: its
        binding unit is the SM's shared-memory data path (ncu: l1tex near
        83%), so that is the roofline reported.  Per 4-site vector an
        overrelaxation update issues 24 16-byte shared-memory loads (own
        spins 3, neighbour rows 15, couplings 6) and 3 16-byte stores: 108 B
        per site update, against the rate of a 16-byte shared-memory load
        stream measured on the device in this run (pt_smem_bandwidth).  The
        FP32 issue view (60 FLOP counted per update) and the
        streaming-equivalent HBM rate are kept beside it."""
        upd = sum(w.n_copies * nt * L ** 3 * (w.n_hb + no)
                  for s, (L, nt, no) in enumerate(zip(w.L, w.n_replicas, nor)) if res_flags[s]) * steps
        if pm["resident"] <= 0 or upd == 0:
            return None
        t = pm["resident"] / 1e3
        n_launch = max(ln["resident"], 1)
        peak_smem = smem_Bps
        n_sm = torch.cuda.get_device_properties(local).multi_processor_count
        peak_alu = n_sm * 128 * 2 * smem_mhz * 1e6
        traffic = ncu_traffic("k_resident", w.name, args.precision) if uniform else None
        return {"bound": "smem", "achieved": upd * 108.0 / t / 1e12, "peak": peak_smem / 1e12, "unit": "TB/s",
                "frac": upd * 108.0 / t / peak_smem, "traffic": traffic,
                "traffic_note": "DRAM bytes per launch (ncu); the replica pool moves once each way per block",
                "kernel": "k_resident / k_resident_cl (sweep block in shared memory, one CTA or a cluster)",
                "peak_source": (f"measured: 16-byte shared-memory load stream on all {n_sm} SMs "
                                f"(pt_smem_bandwidth): {smem_bpc:.1f} B/clock/SM at {smem_mhz:.0f} MHz"),
                "alg_bytes_per_launch": upd * 108.0 / n_launch, "avg_launch_us": t / n_launch * 1e6,
                "effective_hbm_GBps": upd * 36.4 / t / 1e9,
                "alu": {"achieved": upd * 60.0 / t / 1e12, "peak": peak_alu / 1e12, "unit": "TFLOP/s",
                        "frac": upd * 60.0 / t / peak_alu,
                        "peak_source": (f"derived: {n_sm} SMs x 128 FP32 lanes x 2 FLOP at the probe's "
                                        f"{smem_mhz:.0f} MHz, 60 FLOP per update")}}

    dominant = max(("or", "resident"), key=lambda k: prof_ms.get(k, 0.0))
    share = {k: v / max(sum(prof_ms.values()), 1e-9) for k, v in prof_ms.items()}
    streaming = None
    if dominant == "resident":
        roof = resident_roofline(prof_ms, prof_launches, resident, n_prof_steps)
        if uniform and all(resident):
            # the HBM roofline of the streaming half sweep on the same workload
            eng.set_policy("streaming")
            for _ in range(2):
                step(graph=False)
            _, pm2, ln2 = timed(max(2, args.steps // 2), profile=True)
            streaming = or_roofline(pm2, ln2, [False] * w.n_samples, max(2, args.steps // 2))
            eng.set_policy(args.policy)  # back to the tuned paths for the end-to-end pass
    else:
        roof = or_roofline(prof_ms, prof_launches, resident, n_prof_steps)

    # end to end through the public API with host buffers
    R = sum(w.n_copies * n for n in w.n_replicas)
    SNT = sum(w.n_replicas)
    e2e = None
    if not args.no_e2e:
        B_h = torch.from_numpy(np.concatenate(w.betas()).copy()).pin_memory()
        E_h = torch.from_numpy(eps.copy()).pin_memory()
        Hh = torch.empty(R, dtype=torch.float64).pin_memory()
        Qh = torch.empty(SNT * 9, dtype=torch.float64).pin_memory()
        Xh = torch.empty(SNT, dtype=torch.float64).pin_memory()
        Bn, En, Hn, Qn, Xn = (t.numpy() for t in (B_h, E_h, Hh, Qh, Xh))

        def e2e_step():
            eng.set_params(Bn, En)
            eng.cycles(1, w.n_hb, nor[0], mode, measure=False, n_or_samples=nor_samples)
            pt.pt_measure(eng.h, Hn, Qn, Xn)

        for _ in range(2):
            e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        barrier()
        el = time.perf_counter() - t0
        el = sharding.max_over_ranks(el, device="cuda")
        e2e = {"value": sharding.weak_throughput(ups, args.steps, world, el, 1e9), "unit": "updates/ns",
               "h2d_bytes_per_step": int(Bn.nbytes + En.nbytes),
               "d2h_bytes_per_step": int(Hn.nbytes + Qn.nbytes + Xn.nbytes)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, n, el = oracle_cycle_rate(w)
        cpu = {"value": v, "unit": "updates/ns", "cores": 1, "kind": "oracle",
               "sample": f"{n} cycles of one sample (L={w.L[0]}, {w.n_replicas[0]} replicas x {w.n_copies} copies, "
                         f"1 HB + {nor[0]} OR + {mode}) in {el:.1f} s, single thread"}
        va, nc, ela = oracle_rate_all_cores(w)
        cpu["all_cores"] = {"value": va, "unit": "updates/ns", "cores": nc, "kind": "oracle",
                            "sample": f"one process per host core, each cycling its own sample of {w.name} "
                                      f"(L={w.L[0]}) for 12 s; {ela:.1f} s wall"}

    spins_bytes = sum(w.n_copies * nt * L ** 3 * 3 * bpe for L, nt in zip(w.L, w.n_replicas))
    if rank == 0:
        cfg = {"workload": w.name, "samples": w.n_samples, "copies": w.n_copies, "n_hb": w.n_hb,
               "exchange": mode, "eps": w.eps, "precision": args.precision, "policy": args.policy,
               "autotune": None if tune is None else {"choice": [int(c) for c in tune[0]][:8],
                                                      "resident_samples": int(sum(resident))},
               "graph": True, "parallelism": f"samples sharded x{world}",
               "l2": f"inputs larger than L2 ({spins_bytes / 1e6:.0f} MB of spins > 129 MB)"}
        if uniform:
            cfg.update({"L": w.L[0], "replicas": w.n_replicas[0], "n_or": nor[0]})
        else:
            cfg.update({"L": sorted(set(w.L)), "replicas": [min(w.n_replicas), max(w.n_replicas)],
                        "n_or": "5L/4 per sample"})
        line = {
            "metric": "site_updates_per_ns", "value": value, "unit": "updates/ns", "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
            "config": cfg, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "streaming_roofline": streaming,
            "gpu_launches": int(sum(launches.values())), "clocks": clk,
            "kernel_share": share, "kernel_ms_profiled": prof_ms, "kernel_launches_profiled": prof_launches,
        }
        print(json.dumps(line), flush=True)
        if args.log:
            from paper_1006_4247_gb300 import runlog
            runlog.record(args.log, "bench", line["config"], {k: v for k, v in line.items() if k != "config"},
                          engine=runlog.engine_summary(eng))
    eng.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
