"""Multi-process host logic on CPU ranks (gloo, world size 2).

* bench.py's replica aggregation: each rank times its own solves, the job
  time is the MAX over ranks and the throughput counts every rank's solves.
* The row-sharded X^T U exchange of the path (each rank owns a panel of X's
  rows and of U, the partial X_p^T U_p products are summed across ranks):
  equal to the unsharded product and to the oracle's rank-ordered shard sum
  within FP64 rounding.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import synth
        from oracle import enmf_oracle as O
        # replica aggregation: rank r "took" 100 + 50 r ms for 4 solves
        total, value = bench.replica_throughput(100.0 + 50.0 * rank, 4, world)
        # row-sharded X^T U
        X, U0, _ = synth.planted(96, 40, 5, seed=2)
        rows = np.array_split(np.arange(X.shape[0]), world)[rank]
        part = torch.from_numpy(X[rows].T @ U0[rows])
        dist.all_reduce(part, op=dist.ReduceOp.SUM)
        full = X.T @ U0
        shard = O.xtu_sharded(X, U0, world)
        out[rank] = (total, value, float(np.max(np.abs(part.numpy() - full))),
                     float(np.max(np.abs(part.numpy() - shard))), float(np.max(np.abs(full))))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_and_sharded_exchange():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        total, value, err_full, err_shard, scale = out[r]
        assert total == 150.0                       # the slower rank's time
        assert value == pytest.approx(world * 4 / 0.150)
        assert err_full <= 64 * 2.0 ** -52 * scale   # summation order only
        assert err_shard <= 64 * 2.0 ** -52 * scale
