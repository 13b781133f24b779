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


# ---------------------------------------------------------------- batch sharded over ranks
def _oracle_batch_fit(model, offsets, x, y, p0, lb, ub, **kw):
    """CPU stand-in for the per-rank batched GPU fit: the oracle on each fit."""
    from oracle import trf
    nf = len(offsets) - 1
    out = {"popt": [], "pcov": [], "cost": [], "nfev": [], "status": []}
    for k in range(nf):
        a, b = offsets[k], offsets[k + 1]
        r = trf.curve_fit(model, x[a:b], y[a:b], None, p0[k], None if lb is None else lb[k],
                          None if ub is None else ub[k], **kw)
        for key in out:
            out[key].append(r[key])
    return {k: np.asarray(v) for k, v in out.items()}


def _shard_worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2208_12187_gb300 import shard, synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bt = synth.dexp_batch(12, seed=3, m_lo=200, m_hi=2000, dtype=np.float64)
    out = shard.fit_batch_sharded(bt.model, bt.offsets, bt.x, bt.y, bt.p0, rank, world, lb=bt.lb, ub=bt.ub,
                                  fit_fn=_oracle_batch_fit, ftol=1e-10, xtol=1e-10, gtol=1e-10)
    q.put((rank, {k: v.tolist() for k, v in out.items()}))
    dist.destroy_process_group()


def test_lpt_partition_covers_every_fit_once_and_balances_m():
    from paper_2208_12187_gb300 import shard, synth
    sizes = np.diff(synth.dexp_batch(4096, seed=7, dtype=np.float32).offsets)
    for world in (1, 2, 4, 8):
        parts = shard.lpt_partition(sizes, world)
        idx = np.sort(np.concatenate(parts))
        np.testing.assert_array_equal(idx, np.arange(sizes.size))       # every fit exactly once
        loads = np.array([sizes[p].sum() for p in parts])
        assert loads.max() <= sizes.sum() / world + sizes.max()         # LPT's bound
        assert loads.max() / loads.mean() <= 1.01                       # many small fits: near-even
    # a case LPT solves exactly: {7, 5, 4, 3, 3, 2} on 2 ranks -> 12 / 12
    parts = shard.lpt_partition([7, 5, 4, 3, 3, 2], 2)
    assert sorted(int(np.sum(np.array([7, 5, 4, 3, 3, 2])[p])) for p in parts) == [12, 12]
    with pytest.raises(ValueError):
        shard.lpt_partition([1, 2], 0)


def test_two_gloo_ranks_shard_a_batch_like_one_rank():
    """Two gloo ranks each fit their LPT share (a CPU stand-in for the
    per-rank GPU batch) and gather: the gathered results equal the
    single-rank batch's, fit by fit, and both ranks took work."""
    from paper_2208_12187_gb300 import shard, synth
    bt = synth.dexp_batch(12, seed=3, m_lo=200, m_hi=2000, dtype=np.float64)
    one = shard.fit_batch_sharded(bt.model, bt.offsets, bt.x, bt.y, bt.p0, 0, 1, lb=bt.lb, ub=bt.ub,
                                  fit_fn=_oracle_batch_fit, ftol=1e-10, xtol=1e-10, gtol=1e-10)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(2):
        r, out = q.get(timeout=240)
        got[r] = out
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        for k in shard.RESULT_KEYS:
            np.testing.assert_array_equal(np.asarray(got[r][k]), one[k])
        assert set(got[r]["rank"]) == {0, 1}
