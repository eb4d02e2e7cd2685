"""World sharding across ranks (CPU, gloo, world_size 2).

Worlds are independent, so N ranks each step a contiguous world range with no
exchange inside the step; the only collectives are outside the hot path (the
max-over-ranks timing of the benchmark and an optional gather of results). Each
rank here drives the FP64 oracle on its shard with the global world indices as
RNG ids; the gathered result must equal the unsharded run exactly.
"""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2601_22074_b300 import inputs as I

W, STEPS, SEED = 12, 3, 5


def shard(rank: int, world_size: int, n: int):
    """Contiguous world range of `rank` (the partition bench.py's replicas generalise)."""
    per = (n + world_size - 1) // world_size
    return rank * per, min(n, (rank + 1) * per)


def run_worlds(lo, hi):
    from oracle import Oracle
    spec = I.quadruped()
    o = Oracle(spec)
    params = I.randomised_params(spec, W, 3)
    ctrl = I.ctrl_targets(spec, W, STEPS, 4)
    out = []
    for w in range(lo, hi):
        q, v = o.reset(SEED, w)
        a = np.zeros(spec.nv)
        for s in range(STEPS):
            r = o.step(q, v, a, ctrl[s, w], nsub=4, friction_scale=params.friction_scale[w],
                       mass_scale=params.mass_scale[w], kp=params.kp[w], kd=params.kd[w],
                       step_count=s, seed=SEED, world=w)
            q, v, a = r["qpos"], r["qvel"], r["qacc"]
        out.append(np.concatenate([q, v, a]))
    return np.array(out)


def _worker(rank, world_size, port, result_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world_size)
    lo, hi = shard(rank, world_size, W)
    mine = torch.from_numpy(run_worlds(lo, hi))
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world_size)]
    dist.all_gather(sizes, torch.tensor([mine.shape[0]]))
    per = max(int(s) for s in sizes)
    pad = torch.zeros(per, mine.shape[1], dtype=mine.dtype)
    pad[: mine.shape[0]] = mine
    parts = [torch.zeros_like(pad) for _ in range(world_size)]
    dist.all_gather(parts, pad)
    # max-over-ranks reduction, as the benchmark does with its timings
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        full = torch.cat([p[: int(s)] for p, s in zip(parts, sizes)])
        torch.save({"full": full, "max": float(t)}, result_path)
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_rank_sharding_equals_unsharded(tmp_path):
    path = str(tmp_path / "res.pt")
    mp.start_processes(_worker, args=(2, _free_port(), path), nprocs=2, join=True,
                       start_method="spawn")
    res = torch.load(path)
    ref = run_worlds(0, W)
    assert res["max"] == 2.0
    np.testing.assert_array_equal(res["full"].numpy(), ref)


def test_shards_cover_every_world_once():
    for n in (1, 7, 8192, 9216):
        for ws in (1, 2, 4, 8):
            seen = []
            for r in range(ws):
                lo, hi = shard(r, ws, n)
                seen += list(range(lo, hi))
            assert seen == list(range(n))
