"""Run records as JSON lines: one record per measured run, holding the
settings that reproduce it (workload, seeds, precision, sweep paths, step
counter) and what it measured, appended to a file that later analysis reads
line by line.  `bench.py --log PATH` and `python -m
paper_1006_4247_gb300.study ... --log PATH` write them."""
from __future__ import annotations

import json
import os
import time


def engine_summary(eng) -> dict:
    """The engine settings a record needs to be reproduced: lattice sizes and
    replica counts per sample, copies, precision, Philox seed and step, and
    the sweep path of every sample (pt_get_paths codes)."""
    choice, ctas = eng.paths()
    return {"L": [int(v) for v in eng.L], "n_replicas": [int(v) for v in eng.NT], "copies": int(eng.C),
            "precision": eng.precision, "seed": int(eng.seed), "step": int(eng.step),
            "paths": [int(v) for v in choice], "ctas_per_replica": [int(v) for v in ctas]}


def record(path: str, kind: str, config: dict, results: dict, engine: dict | None = None) -> dict:
    """Append one record {time, kind, config, results[, engine]} to `path`
    (created with its directory if missing) and return it."""
    rec = {"time": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()), "kind": kind, "config": config,
           "results": results}
    if engine is not None:
        rec["engine"] = engine
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    with open(path, "a") as fh:
        fh.write(json.dumps(rec, sort_keys=True) + "\n")
    return rec


def read(path: str, kind: str | None = None) -> list:
    """All records of the file (of one kind if given), in the order written."""
    out = []
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if line:
                r = json.loads(line)
                if kind is None or r.get("kind") == kind:
                    out.append(r)
    return out
