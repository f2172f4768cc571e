"""Write tests/golden/stats_L4_R8.json: per-run averages of the FP64 oracle
for the long-run statistical parity test (calls only the oracle).

Workload: L = 4 periodic lattice, Gaussian couplings from
paper_1006_4247_gb300.workloads.couplings(4, 1), 8 inverse temperatures
linear in [2.5, 8.0], two copies, 1 heat-bath + 3 overrelaxation sweeps and
one tempering update per cycle, 1000 cycles of which the first 200 are
discarded; 96 independent runs (seeds 9000..9095) per exchange mode
(standard; decimation; cooling/heating with eps = 0.05).

    python tests/golden/make_stats_L4.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as orc  # noqa: E402
from paper_1006_4247_gb300 import workloads as W  # noqa: E402

L, NT, CYCLES, BURN, RUNS = 4, 8, 1000, 200, 96
MODES = {"plain": (0, 0.0), "decimation": (1, 0.0), "coolheat": (2, 0.05)}


def main():
    betas = W.linear_betas(NT, 2.5, 8.0)
    J = W.couplings(L, 1).astype(np.float64)
    out = {"L": L, "NT": NT, "cycles": CYCLES, "burn": BURN, "betas": betas.tolist(), "modes": {}}
    for name, (mode, eps) in MODES.items():
        H, C, A = [], [], []
        for r in range(RUNS):
            run = orc.Run(L, J, betas, n_copies=2, seed=9000 + r, eps=eps)
            Hs, chis, _ = run.cycles(CYCLES, n_hb=1, n_or=3, mode=mode)
            H.append(Hs[BURN:].mean(axis=(0, 1)).tolist())
            C.append(chis[BURN:].mean(axis=0).tolist())
            A.append((run.acc / np.maximum(run.prop, 1)).mean(axis=0).tolist())
        out["modes"][name] = {"eps": eps, "H": H, "chi": C, "acc": A}
        print(name, "done", flush=True)
    with open(os.path.join(HERE, "stats_L4_R8.json"), "w") as fh:
        json.dump(out, fh)


if __name__ == "__main__":
    main()
