"""Host logic of multi-GPU runs, checked with two CPU ranks over gloo: every
rank gets disjoint coupling seeds and its own Philox seed (no data-path
exchange), the timing takes the maximum over ranks after a barrier, and the
throughput counts the work of all ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1006_4247_gb300 import sharding  # noqa: E402
from paper_1006_4247_gb300 import workloads as W  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = W.WORKLOADS["L16_R24_S64"]()
        w.j_seed0 = sharding.coupling_seed0(w.j_seed0, rank)
        seeds = [w.j_seed0 + s for s in range(w.n_samples)]
        J0 = w.couplings()[0]
        gathered = [None] * world
        dist.all_gather_object(gathered, {"seeds": seeds, "engine_seed": sharding.engine_seed(rank),
                                          "J0_sum": float(np.asarray(J0, np.float64).sum())})
        sharding.barrier()
        elapsed = 1.0 + 0.5 * rank  # rank 1 is the slow one
        t = sharding.max_over_ranks(elapsed)
        v = sharding.weak_throughput(100.0, 4, world, t, 1.0)
        np.save(os.path.join(out_dir, f"r{rank}.npy"),
                np.array([t, v, len(set(gathered[0]["seeds"]) & set(gathered[1]["seeds"])),
                          gathered[0]["engine_seed"], gathered[1]["engine_seed"],
                          gathered[0]["J0_sum"] != gathered[1]["J0_sum"]], np.float64))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_samples_and_time_by_maximum(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for rank in range(world):
        t, v, overlap, es0, es1, differ = np.load(tmp_path / f"r{rank}.npy")
        assert t == 1.5                      # the maximum over ranks, seen by every rank
        assert v == pytest.approx(100.0 * 4 * 2 / 1.5)
        assert overlap == 0                  # disjoint coupling seeds
        assert es0 != es1                    # distinct Philox streams
        assert differ                        # different couplings


def test_single_process_paths_need_no_group():
    assert not dist.is_initialized()
    assert sharding.max_over_ranks(2.5) == 2.5
    sharding.barrier()
    assert sharding.weak_throughput(10.0, 3, 1, 2.0, 1.0) == 15.0
    with pytest.raises(ValueError):
        sharding.weak_throughput(10.0, 3, 1, 0.0, 1.0)
    assert sharding.coupling_seed0(100, 0) == 100 and sharding.coupling_seed0(100, 3) == 300100
