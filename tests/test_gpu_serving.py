"""Serving by continuous batching (gbfit_server_*).

A stream of requests of three models and many sizes is served through a
small pool (forcing queueing) and few slots; more requests arrive while
others are running.  Each result must equal, bit for bit, the same fit run
alone through gbfit_curve_fit with the same reduction shape (a served fit's
shape depends only on its own m, through the tile table),
and match the FP64 oracle: plain 1e-8 relative on popt; mixed by the per-fit
criterion of oracle_checks (popt within 1e-6 where the oracle's popt is
determined to that level, else no higher cost than the oracle's).  The mixed
stream includes near-degenerate double exponentials (t2 within 30 % of t1),
whose Gram is ill-conditioned enough for the precision guard to move them to
FP64 passes while they share launches with FP32 fits.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle_checks
from oracle import trf
from paper_2208_12187_gb300 import build, gbfit, synth

pytestmark = pytest.mark.gpu
TOL = dict(ftol=1e-10, xtol=1e-10, gtol=1e-10)


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return gbfit.load()


def _requests(dtype, degenerate=False):
    rng = np.random.default_rng(5)
    reqs = []
    for k in range(18):
        kind = k % 3
        m = int(np.exp(rng.uniform(np.log(2e3), np.log(2e5))))
        if kind == 0:
            pr = synth.gauss1d(m, seed=k, with_sigma=bool(k % 2), dtype=dtype)
        elif kind == 1 and degenerate and k % 2 == 0:
            t1 = 1.0 + 0.2 * k
            pr = synth.dexp(m, seed=k, truth=[4.0, t1, 6.0, t1 * (1.15 + 0.01 * k), 0.5], dtype=dtype)
        elif kind == 1:
            pr = synth.dexp(m, seed=k, truth=[4.0, 0.5 + 0.1 * k, 6.0, 5.0 + k, 0.5], dtype=dtype)
        else:
            W = int(np.sqrt(m))
            pr = synth.gauss2d_grid(W, seed=k, dtype=dtype)
        reqs.append(pr)
    return reqs


@pytest.mark.parametrize("precision,dtype,rel", [("mixed", np.float32, 1e-6), ("fp64", np.float64, 1e-8)])
def test_served_equals_alone_and_oracle(precision, dtype, rel):
    reqs = _requests(dtype, degenerate=precision == "mixed")
    srv = gbfit.Server(hbm_budget_bytes=8 << 20, max_slots=5, precision=precision, rounds_per_step=3)
    tickets = {}

    def submit(k):
        pr = reqs[k]
        x = None if pr.layout == synth.LAYOUT_GRID else pr.x
        tickets[srv.submit(pr.model, x, pr.y, pr.p0, sigma=pr.sigma, lb=pr.lb, ub=pr.ub, grid_wh=pr.grid_wh,
                           tag=k, **TOL)] = k

    for k in range(8):
        submit(k)
    results = {}
    steps = 0
    nxt = 8
    while len(results) < len(reqs):
        active, queued = srv.step()
        steps += 1
        if nxt < len(reqs):              # arrivals while others run
            submit(nxt)
            nxt += 1
        for r in srv.poll():
            results[r["tag"]] = r
        assert steps < 10000
    srv.close()
    for k, pr in enumerate(reqs):
        r = results[k]
        assert r["status"] == 0 and r["fit_status"] in (1, 2, 3, 4)
        assert r["t_submit"] <= r["t_admit"] <= r["t_done"]
        x = None if pr.layout == synth.LAYOUT_GRID else torch.as_tensor(pr.x).cuda()
        tp, gt = gbfit.tune_shape(pr.model, precision, pr.m)     # the shape the server gave this fit
        alone = gbfit.curve_fit(pr.model, x, torch.as_tensor(pr.y).cuda(), pr.p0,
                                sigma=None if pr.sigma is None else torch.as_tensor(pr.sigma).cuda(),
                                lb=pr.lb, ub=pr.ub, grid_wh=pr.grid_wh, precision=precision,
                                tile_points=tp, group_tiles=gt, **TOL)
        np.testing.assert_array_equal(r["popt"], alone["popt"])
        assert r["nfev"] == alone["nfev"]
        ref = trf.curve_fit_problem(pr, **TOL)
        if precision == "mixed":
            oracle_checks.check_mixed(pr.astype(np.float64), r["popt"], ref, TOL, rel=rel)
        else:
            err = np.max(np.abs(r["popt"] - ref["popt"]) / np.maximum(np.abs(ref["popt"]), 1.0))
            assert err <= rel, (k, err)


def test_budget_refusal():
    srv = gbfit.Server(hbm_budget_bytes=1 << 20, max_slots=2)
    pr = synth.gauss1d(300_000, seed=1, dtype=np.float32)
    with pytest.raises(gbfit.GbfitError) as e:
        srv.submit(pr.model, pr.x, pr.y, pr.p0)
    assert e.value.code == gbfit.E_BUDGET
    srv.close()
