"""Multi-rank bookkeeping of bench.py on CPU ranks (gloo, world size 2).

Value sets are independent, so the GPU path shards by instance with no
collective in the data path; what needs checking is the host logic: every
rank builds its own value sets (distinct seeds, identical to what a single
process builds for that rank), each rank's systems solve correctly, and the
whole-job throughput uses the slowest rank's time; the plan is analyzed
once, on rank 0, and reaches the other ranks through its file."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from oracle import oracle as O
    work, _ = bench.make_workload("tiny", rank)
    (p, B), = work
    res = []
    for i in range(B):
        r = O.refactor_solve(p, i)
        res.append(np.linalg.norm(O.symv(r.K, r.x) - p.b[i]) / np.linalg.norm(p.b[i]))
    local_ms = 10.0 * (rank + 1)
    value, max_ms = bench.aggregate_value(B, 4, local_ms, dist)
    # the plan is analyzed once (rank 0) and replicated through its file
    from paper_2110_12865_gb300 import ssco as S
    pl, = bench.shared_plans(work, S.FP32_REFINE, rank, world, dist, S)
    own = S.Plan(p, precision=S.FP32_REFINE, batch=B)
    same_plan = pl.info == own.info and all(np.array_equal(pl.export(k), own.export(k)) for k in range(15))
    w = torch.tensor(p.vals[0][:8].copy())
    gathered = [torch.zeros_like(w) for _ in range(world)]
    dist.all_gather(gathered, w)
    out[rank] = {"value": value, "max_ms": max_ms, "res": max(res), "same_plan": same_plan,
                 "first_vals": [g.numpy().tolist() for g in gathered]}
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    from paper_2110_12865_gb300 import build
    build.build()
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        out = dict(out)
    import bench
    for rank in range(world):
        o = out[rank]
        assert o["max_ms"] == 20.0                       # the slowest rank's time
        assert abs(o["value"] - 3 * world * 4 / 0.020) < 1e-9
        assert o["res"] < 1e-12
        assert o["same_plan"]                             # the replicated plan is the analyzed one
        work, _ = bench.make_workload("tiny", rank)       # same data as a single process builds
        assert np.allclose(out[0]["first_vals"][rank], work[0][0].vals[0][:8])
    assert not np.allclose(out[0]["first_vals"][0], out[0]["first_vals"][1])  # distinct value sets


def test_oracle_timing_on_all_host_cores():
    """The CPU baseline deals its systems to one spawned process per host
    core (largest first, least loaded core); each process runs only the
    numeric oracle after a common start, and the wall time is the slowest
    process's, so it is at most the summed busy time."""
    import bench
    work, _ = bench.make_workload("tiny", 0)
    items = bench.oracle_sample(work) * 3
    wall, busy, procs, limit = bench.time_oracle_all_cores(items)
    assert 1 <= procs <= min(len(os.sched_getaffinity(0)), len(items))
    assert 0 < wall <= busy + 1e-9
    assert limit >= 600.0


def test_oracle_timing_fails_fast_when_a_worker_dies():
    """A worker whose oracle call raises (here: a system of an unknown kind)
    ends the CPU baseline with RuntimeError within seconds, and no worker
    process is left behind (the others were waiting at the start barrier)."""
    import multiprocessing as mp
    import time
    import bench
    work, _ = bench.make_workload("tiny", 0)
    items = bench.oracle_sample(work) * 2
    bad = bench._one_system(*items[0])
    bad["kind"] = 99                                 # neither A^T W A nor element blocks
    bad["name"] = "broken"
    items = [(bad, 0)] + items
    t0 = time.monotonic()
    with pytest.raises(RuntimeError):
        bench.time_oracle_all_cores(items, limit_s=60.0)
    assert time.monotonic() - t0 < 30.0
    assert not [c for c in mp.active_children() if c.is_alive()]
