"""The N > 1 host path of bench.py on CPU: two gloo ranks, no GPU.

Fits are independent problems (weak scaling): each rank fits its own seeded
problem and the only cross-rank traffic is host-side (barriers, the max of
the ranks' times and the sum of their points); the reference arm runs on
rank 0 only, the other ranks return without work.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        steps, warmup, ref_nfev, gpus = 1, 0, 1, world

    r, _, w = bench.dist_setup(Args())
    mx = bench.allreduce([float(r + 1), 10.0 * r], "max", w)
    sm = bench.allreduce([float(r + 1)], "sum", w)
    bench.barrier(w)
    pr = bench.make_problem(r)
    ref = bench.run_reference(Args(), r, w)
    bench.barrier(w)
    q.put((r, mx, sm, float(np.sum(pr.y[:1000])), None if ref is None else (ref["impl"], ref["unit"])))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_and_partition():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(2):
        r, mx, sm, ysum, ref = q.get(timeout=240)
        out[r] = (mx, sm, ysum, ref)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        assert out[r][0] == [2.0, 10.0]          # max over ranks
        assert out[r][1] == [3.0]                # sum over ranks
    assert out[0][2] != out[1][2]                # each rank draws its own problem
    assert out[0][3] == ("reference", "point-iters/s")
    assert out[1][3] is None                     # only rank 0 runs the reference arm
