"""Write tests/golden/stats_L16_R24.json and tests/golden/stats_L32_R48.json:
per-run averages of the FP64 oracle for the long-run statistical parity test
at the sizes of the benchmark batches (calls only the oracle).

  L = 16: Gaussian couplings paper_1006_4247_gb300.workloads.couplings(16, 100)
          (the first sample of the 64-sample batch), 24 inverse temperatures
          linear in [2.0, 8.0], two copies, 1 heat-bath + 20 overrelaxation
          sweeps (5L/4) and one cooling/heating update (eps = 0.017 rounded
          to float, the value the engine holds) per cycle; 150 cycles of
          which the first 50 are discarded; 32 independent runs (seeds
          9100..9131).
  L = 32: couplings(32, 200) (the first sample of the 16-sample batch), 48
          inverse temperatures linear in [2.0, 8.0], two copies, 1 + 40 sweeps
          and one decimation update per cycle; 40 cycles of which the first 10
          are discarded; 24 independent runs (seeds 9200..9223).
  L = 16 with the standard swap (stats_L16_R24_plain.json, seeds 9300..9331)
          and with decimation (stats_L16_R24_decimation.json, seeds
          9400..9431), otherwise as the first case.

Every run starts from spins uniform on the sphere (its own Philox stream), so
the per-run averages are independent draws of the same random variable for
the oracle and for the engine, whether or not the chains have reached
equilibrium by then.  Runs are spread over the host's cores (one process per
run, started with spawn); about 4 min (L = 16) and 20 min (L = 32) on 8 cores.

    python tests/golden/make_stats_large.py [16] [32] [161] [162]
"""
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

CASES = {
    16: {"file": "stats_L16_R24.json", "NT": 24, "j_seed": 100, "n_or": 20,
         "mode": ("coolheat", 2, float(np.float32(0.017))), "cycles": 150, "burn": 50, "runs": 32, "seed0": 9100},
    32: {"file": "stats_L32_R48.json", "NT": 48, "j_seed": 200, "n_or": 40, "mode": ("decimation", 1, 0.0),
         "cycles": 40, "burn": 10, "runs": 24, "seed0": 9200},
    # configuration 2's other exchanges: the standard swap and decimation
    161: {"L": 16, "file": "stats_L16_R24_plain.json", "NT": 24, "j_seed": 100, "n_or": 20,
          "mode": ("plain", 0, 0.0), "cycles": 150, "burn": 50, "runs": 32, "seed0": 9300},
    162: {"L": 16, "file": "stats_L16_R24_decimation.json", "NT": 24, "j_seed": 100, "n_or": 20,
          "mode": ("decimation", 1, 0.0), "cycles": 150, "burn": 50, "runs": 32, "seed0": 9400},
}


def one_run(job):
    key, r = job
    import oracle as orc
    from paper_1006_4247_gb300 import workloads as W
    c = CASES[key]
    L = c.get("L", key)
    betas = W.linear_betas(c["NT"], 2.0, 8.0)
    J = W.couplings(L, c["j_seed"]).astype(np.float64)
    name, mode, eps = c["mode"]
    run = orc.Run(L, J, betas, n_copies=2, seed=c["seed0"] + r, eps=eps)
    run.cycles(c["burn"], n_hb=1, n_or=c["n_or"], mode=mode, record=False)
    a0, p0 = run.acc.copy(), run.prop.copy()
    Hs, chis, _ = run.cycles(c["cycles"] - c["burn"], n_hb=1, n_or=c["n_or"], mode=mode)
    # per run: <H>(beta) over both copies, <chi>(beta), and the acceptance of
    # every pair over the kept cycles (counts after the burn-in minus before)
    return (Hs.mean(axis=(0, 1)).tolist(), chis.mean(axis=0).tolist(),
            ((run.acc - a0) / np.maximum(run.prop - p0, 1)).mean(axis=0).tolist())


def main(sizes):
    import oracle as orc
    orc.build()
    ctx = mp.get_context("spawn")
    for key in sizes:
        c = CASES[key]
        L = c.get("L", key)
        t0 = time.time()
        with ctx.Pool(os.cpu_count() or 1) as pool:
            res = pool.map(one_run, [(key, r) for r in range(c["runs"])])
        from paper_1006_4247_gb300 import workloads as W
        name, mode, eps = c["mode"]
        out = {"L": L, "NT": c["NT"], "j_seed": c["j_seed"], "n_hb": 1, "n_or": c["n_or"], "cycles": c["cycles"],
               "burn": c["burn"], "betas": W.linear_betas(c["NT"], 2.0, 8.0).tolist(), "mode": name, "eps": eps,
               "seeds": [c["seed0"] + r for r in range(c["runs"])],
               "H": [x[0] for x in res], "chi": [x[1] for x in res], "acc": [x[2] for x in res]}
        with open(os.path.join(HERE, c["file"]), "w") as fh:
            json.dump(out, fh)
        print(f"L={L}: {c['runs']} runs in {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or list(CASES))
