"""Independent fits spread over ranks (one process per GPU).

Batched and served fits are independent problems, so the path shards with no
data-path collective: each rank fits a subset of the fits on its own GPU
(one gbfit_curve_fit_batch launch), and the per-fit results meet on the host
afterwards.  The subsets balance the work, taken as proportional to each
fit's number of points m, by the longest-processing-time-first rule: fits in
decreasing m, each to the rank with the least m so far (ties: the lower rank;
the result is within 4/3 of the optimal largest load).

The fitting call and the gather are parameters, so that the host logic runs
without a GPU (tests drive it through gloo ranks with a CPU stand-in).
"""
from __future__ import annotations

from typing import Callable, Optional, Sequence

import numpy as np


def lpt_partition(sizes: Sequence[int], world: int) -> list[np.ndarray]:
    """Indices of the fits each rank takes, each list in increasing index order."""
    sizes = np.asarray(sizes, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    if np.any(sizes < 0):
        raise ValueError("sizes must be >= 0")
    order = np.lexsort((np.arange(sizes.size), -sizes))   # decreasing size, then index
    load = np.zeros(world, dtype=np.int64)
    owner = np.empty(sizes.size, dtype=np.int64)
    for k in order:
        r = int(np.argmin(load))                              # first rank of least load
        owner[k] = r
        load[r] += sizes[k]
    return [np.flatnonzero(owner == r) for r in range(world)]


def sub_batch(offsets: np.ndarray, idx: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Offsets of the sub-batch made of fits idx (in that order) and the
    point indices of the full batch it takes, concatenated."""
    offsets = np.asarray(offsets, dtype=np.int64)
    m = offsets[1:] - offsets[:-1]
    sub_off = np.zeros(idx.size + 1, dtype=np.int64)
    sub_off[1:] = np.cumsum(m[idx])
    pts = np.concatenate([np.arange(offsets[k], offsets[k + 1]) for k in idx]) if idx.size else np.zeros(0, np.int64)
    return sub_off, pts


RESULT_KEYS = ("popt", "pcov", "cost", "nfev", "status")


def fit_batch_sharded(model: int, offsets, xdata: np.ndarray, ydata: np.ndarray, p0, rank: int, world: int,
                      lb=None, ub=None, fit_fn: Optional[Callable] = None,
                      gather_fn: Optional[Callable] = None, **kw) -> dict:
    """Fit this rank's share of a batch and return the whole batch's results
    (every rank gets them, in the batch's order).

    xdata, ydata: host arrays of the whole batch (each rank slices its share);
    fit_fn(model, offsets, x, y, p0, lb, ub, **kw) -> dict of RESULT_KEYS
    (default: gbfit.curve_fit_batch on this rank's GPU); gather_fn(obj) ->
    list of every rank's obj (default: torch.distributed.all_gather_object;
    with world == 1 no gather is done)."""
    offsets = np.asarray(offsets, dtype=np.int64)
    nf = offsets.size - 1
    n = np.asarray(p0).reshape(nf, -1).shape[1]
    p0 = np.asarray(p0, dtype=np.float64).reshape(nf, n)
    lb = None if lb is None else np.broadcast_to(np.asarray(lb, np.float64), (nf, n))
    ub = None if ub is None else np.broadcast_to(np.asarray(ub, np.float64), (nf, n))
    parts = lpt_partition(offsets[1:] - offsets[:-1], world)
    mine = parts[rank]
    if fit_fn is None:
        fit_fn = _gpu_fit
    res = None
    if mine.size:
        sub_off, pts = sub_batch(offsets, mine)
        res = fit_fn(model, sub_off, np.ascontiguousarray(xdata[pts]), np.ascontiguousarray(ydata[pts]), p0[mine],
                     None if lb is None else lb[mine], None if ub is None else ub[mine], **kw)
        res = {k: np.asarray(res[k]) for k in RESULT_KEYS}
    shares = [(mine, res)] if world == 1 else (gather_fn or _all_gather)((mine, res))
    out = {"popt": np.zeros((nf, n)), "pcov": np.zeros((nf, n, n)), "cost": np.zeros(nf),
           "nfev": np.zeros(nf, dtype=np.int32), "status": np.zeros(nf, dtype=np.int32),
           "rank": np.full(nf, -1, dtype=np.int32)}
    for r, (idx, part) in enumerate(shares):
        if part is None:
            continue
        for k in RESULT_KEYS:
            out[k][idx] = part[k]
        out["rank"][idx] = r
    return out


def _gpu_fit(model, offsets, x, y, p0, lb, ub, **kw):
    import torch
    from . import gbfit
    xt = torch.as_tensor(x).cuda()
    yt = torch.as_tensor(y).cuda()
    return gbfit.curve_fit_batch(model, offsets, xt, yt, p0, lb=lb, ub=ub, **kw)


def _all_gather(obj):
    import torch.distributed as dist
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, obj)
    return out
