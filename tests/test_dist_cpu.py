"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

The batched form partitions into independent (structure, candidate) items: with N GPUs
every rank evaluates its own batch and only the timing crosses ranks (barrier + max over
ranks).  These tests run that host logic as two gloo processes; no GPU is involved.
"""
import json
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, outdir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2601_19034_gb300 import workloads as wl
    w, r, _ = bench._dist()
    step_ms = 10.0 + 5.0 * rank                         # a slower rank sets the job's time
    dist.barrier()
    ms = bench._reduce_max(step_ms)
    systems, hp, params, elec = wl.config_llzo_batch(seed=bench._batch_seed(rank), n_struct=3, n_candidates=2)
    res = {"world": w, "rank": r, "ms": ms, "seed": bench._batch_seed(rank),
           "sizes": [int(s.n_atoms) for s in systems], "first": systems[0].positions[:4].tolist()}
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_and_independent_batches(tmp_path):
    world, port = 2, _free_port()
    mp.spawn(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    assert [x["rank"] for x in res] == [0, 1] and all(x["world"] == 2 for x in res)
    # max over ranks: every rank reports the slowest rank's time
    assert all(x["ms"] == 15.0 for x in res)
    # each rank evaluates its own batch: distinct seeds, distinct structures, LLZO sizes
    assert res[0]["seed"] != res[1]["seed"]
    assert not np.allclose(res[0]["first"], res[1]["first"])
    for x in res:
        assert all(s in (192, 384, 768, 1536) for s in x["sizes"])


def test_single_process_reduce_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._reduce_max(3.5) == 3.5
    assert bench._batch_seed(0) == 1003   # rank 0 keeps the single-GPU workload
