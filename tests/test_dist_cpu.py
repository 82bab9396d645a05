"""Multi-rank host logic on CPU (gloo, world size 2): bench.py and the distributed SNES step.

The batched form partitions into independent (structure, candidate) items: with N GPUs
every rank evaluates its own batch and only the timing crosses ranks (barrier + max over
ranks).  The distributed SNES step shards the population instead (each rank scores its
candidates on every structure) and has one real exchange: the all-gather of the C losses,
after which every rank takes the same update from the same seeded deviates.  These tests
run that host logic as two gloo processes; no GPU is involved.
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


def _snes_worker(rank, world, port, outdir):
    """One distributed SNES iteration: each rank scores its candidate shard, the losses are
    all-gathered, every rank applies the same update (the oracle's update stands in for the
    device kernel, which needs a GPU)."""
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import training as tr
    from paper_2601_19034_gb300.qnep import candidate_shard, gather_losses, snes_noise
    n_cand, n_par = 7, 11
    rng = np.random.default_rng(3)                      # the same problem on every rank
    a, target = rng.uniform(0.5, 2.0, n_par), rng.normal(size=n_par)
    mu, sigma = np.full(n_par, 2.0), np.ones(n_par)
    for step in range(3):
        noise = snes_noise(n_cand, n_par, step, seed=100, device="cpu").double().numpy()
        c0, c1 = candidate_shard(n_cand, world, rank)
        z = tr.sample(mu, sigma, noise[c0:c1])
        local = torch.tensor(((z - target) ** 2 * a).sum(1))
        losses = gather_losses(local, n_cand).numpy()
        mu, sigma = tr.update(mu, sigma, noise, losses)
    with open(os.path.join(outdir, f"snes{rank}.json"), "w") as f:
        json.dump({"shard": [c0, c1], "mu": mu.tolist(), "sigma": sigma.tolist(), "losses": losses.tolist()}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_snes_iteration_matches_one_process(tmp_path):
    world, port = 2, _free_port()
    mp.spawn(_snes_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"snes{r}.json")) for r in range(world)]
    assert res[0]["shard"] == [0, 4] and res[1]["shard"] == [4, 7]      # uneven shards cover the population
    for key in ("mu", "sigma", "losses"):
        np.testing.assert_array_equal(res[0][key], res[1][key])         # every rank takes the same step
    # the same three iterations in one process, every candidate scored locally
    sys.path.insert(0, ROOT)
    from oracle import training as tr
    from paper_2601_19034_gb300.qnep import snes_noise
    rng = np.random.default_rng(3)
    a, target = rng.uniform(0.5, 2.0, 11), rng.normal(size=11)
    mu, sigma = np.full(11, 2.0), np.ones(11)
    for step in range(3):
        noise = snes_noise(7, 11, step, seed=100, device="cpu").double().numpy()
        f = ((tr.sample(mu, sigma, noise) - target) ** 2 * a).sum(1)
        mu, sigma = tr.update(mu, sigma, noise, f)
    np.testing.assert_allclose(res[0]["mu"], mu, rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(res[0]["sigma"], sigma, rtol=1e-15, atol=1e-15)


def test_candidate_shards_partition_the_population():
    sys.path.insert(0, ROOT)
    from paper_2601_19034_gb300.qnep import candidate_shard
    for n in (1, 7, 64, 100):
        for world in (1, 2, 3, 8):
            spans = [candidate_shard(n, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[r][1] == spans[r + 1][0] for r in range(world - 1))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
