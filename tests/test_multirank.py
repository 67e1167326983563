"""The multi-GPU path of the benchmark, run as two gloo ranks on CPU: every rank takes its
own seeded batch (independent scenes, no data-path collective), the timing is the maximum
over ranks, and the reference arm runs on rank 0 only."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch
    import bench
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = bench.make_problem("batched", rank, scenes=2)
    o = oracle.OracleScene(p.scenes[0], p.options)
    o.step()
    first_body = o.bodies_all()[0, 4:7].copy()
    t_ms = 10.0 * (rank + 1)                 # a stand-in for the rank's timed region
    tt = torch.tensor([t_ms])
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    pos = torch.tensor(first_body)
    gathered = [torch.zeros(3, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(gathered, pos)           # test-only: compare the ranks' batches
    out[rank] = (float(tt.item()), bench.whole_job_rate(world, 5, float(tt.item())),
                 [g.numpy().tolist() for g in gathered])
    dist.destroy_process_group()


def test_two_ranks_shard_independent_batches():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    t0, v0, g0 = res[0]
    t1, v1, g1 = res[1]
    assert t0 == t1 == 20.0                  # max over ranks
    assert v0 == v1 == pytest.approx(2 * 5 / 0.020)
    assert not np.allclose(g0[0], g0[1])     # different seeded batches per rank


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import argparse
    import bench
    args = argparse.Namespace(workload="batched", robots=1, scenes=2, warmup=3, steps=1,
                              reference_seconds=1.0, reference_scenes=0)
    assert bench.run_reference(args, rank=1, world=2) == 0
    assert capsys.readouterr().out == ""
