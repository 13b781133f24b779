"""Failure detection and recovery without a GPU fault.

* Bounded device waits running out: gbfit_options.wait_limit_s shortens the
  loop kernel's grid-wide waits (round barrier, owner wait, queue-mode idle
  wait) to 1 microsecond, shorter than any trust-region step, so a normal fit
  gives up: the call returns GBFIT_E_TIMEOUT (nothing traps, nothing waits
  without a limit) and the next ordinary call on the same context gives the
  oracle's result.
* Serving: cancellation of a queued and of a resident request between steps
  (their records carry GBFIT_E_CANCELLED, the others finish normally), and a
  snapshot of a resident fit resumed in another server gives bitwise the
  result of the uninterrupted fit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


def _relerr(a, b):
    return float(np.max(np.abs(np.asarray(a) - b) / np.maximum(np.abs(b), 1.0)))


def test_single_fit_wait_limit_times_out_then_context_is_usable():
    pr = synth.gauss1d(200_000, seed=3)
    x, y = torch.as_tensor(pr.x).cuda(), torch.as_tensor(pr.y).cuda()
    for prec in ("fp64", "mixed"):
        xx, yy = (x, y) if prec == "fp64" else (x.float(), y.float())
        with pytest.raises(gbfit.GbfitError) as e:
            gbfit.curve_fit(pr.model, xx, yy, pr.p0, precision=prec, wait_limit_s=1e-6, **TOL)
        assert e.value.code == gbfit.E_TIMEOUT
    out = gbfit.curve_fit(pr.model, x, y, pr.p0, precision="fp64", **TOL)
    ref = trf.curve_fit_problem(pr, **TOL)
    assert _relerr(out["popt"], ref["popt"]) <= 1e-8 and out["nfev"] == ref["nfev"]


def test_batch_wait_limit_times_out_then_context_is_usable():
    bt = synth.dexp_batch(16, seed=31, m_lo=2000, m_hi=20_000, dtype=np.float64)
    x, y = torch.as_tensor(bt.x).cuda(), torch.as_tensor(bt.y).cuda()
    kw = dict(lb=bt.lb, ub=bt.ub, precision="fp64", **TOL)
    with pytest.raises(gbfit.GbfitError) as e:
        gbfit.curve_fit_batch(bt.model, bt.offsets, x, y, bt.p0, wait_limit_s=1e-6, **kw)
    assert e.value.code == gbfit.E_TIMEOUT
    out = gbfit.curve_fit_batch(bt.model, bt.offsets, x, y, bt.p0, **kw)
    for k in (0, 9):
        ref = trf.curve_fit_problem(bt.fit(k), **TOL)
        assert _relerr(out["popt"][k], ref["popt"]) <= 1e-8 and out["nfev"][k] == ref["nfev"]


def test_wait_limit_option_checked():
    pr = synth.gauss1d(1000, seed=1)
    with pytest.raises(gbfit.GbfitError) as e:
        gbfit.curve_fit(pr.model, torch.as_tensor(pr.x).cuda(), torch.as_tensor(pr.y).cuda(), pr.p0,
                        precision="fp64", wait_limit_s=float("nan"))
    assert e.value.code == gbfit.E_INVALID_ARG


def _submit(srv, pr, tag, **kw):
    return srv.submit(pr.model, pr.x, pr.y, pr.p0, sigma=pr.sigma, lb=pr.lb, ub=pr.ub, tag=tag, **TOL, **kw)


def _drain(srv, want, limit=100_000):
    got = {}
    steps = 0
    while len(got) < want:
        srv.step()
        for r in srv.poll():
            got[r["tag"]] = r
        steps += 1
        assert steps < limit
    return got


def test_cancel_queued_and_resident_requests():
    probs = [synth.gauss1d(50_000, seed=40 + k, dtype=np.float32) for k in range(6)]
    srv = gbfit.Server(hbm_budget_bytes=64 << 20, max_slots=2, precision="mixed", rounds_per_step=1)
    tickets = [_submit(srv, pr, k) for k, pr in enumerate(probs)]
    srv.cancel(tickets[5])                      # still queued: never started
    srv.step()                                  # requests 0 and 1 resident, one evaluation done
    srv.cancel(tickets[0])                      # resident
    with pytest.raises(gbfit.GbfitError) as e:
        srv.cancel(12345)
    assert e.value.code == gbfit.E_INVALID_ARG
    got = _drain(srv, 6)
    srv.close()
    assert got[5]["status"] == gbfit.E_CANCELLED and got[5]["nfev"] == 0
    np.testing.assert_array_equal(got[5]["popt"], probs[5].p0)
    assert got[0]["status"] == gbfit.E_CANCELLED and got[0]["nfev"] >= 1
    for k in (1, 2, 3, 4):
        assert got[k]["status"] == 0 and got[k]["fit_status"] in (1, 2, 3, 4)
        alone = gbfit.curve_fit(probs[k].model, probs[k].x, probs[k].y, probs[k].p0, precision="mixed", **TOL)
        assert _relerr(got[k]["popt"], alone["popt"]) <= 1e-6


@pytest.mark.parametrize("precision,dtype", [("mixed", np.float32), ("fp64", np.float64)])
def test_snapshot_resume_gives_the_uninterrupted_result(precision, dtype):
    pr = synth.dexp(30_000, seed=44, dtype=dtype)
    # uninterrupted
    srv = gbfit.Server(hbm_budget_bytes=64 << 20, max_slots=4, precision=precision, rounds_per_step=1)
    _submit(srv, pr, 0)
    ref = _drain(srv, 1)[0]
    srv.close()
    assert ref["nfev"] >= 4
    # interrupted after three evaluations, resumed in another server
    srv = gbfit.Server(hbm_budget_bytes=64 << 20, max_slots=4, precision=precision, rounds_per_step=1)
    t = _submit(srv, pr, 0)
    for _ in range(3):
        srv.step()
    snap = srv.snapshot(t)
    srv.cancel(t)
    part = _drain(srv, 1)[0]
    srv.close()
    assert part["status"] == gbfit.E_CANCELLED and 1 <= part["nfev"] < ref["nfev"]
    srv = gbfit.Server(hbm_budget_bytes=64 << 20, max_slots=4, precision=precision, rounds_per_step=1)
    _submit(srv, pr, 1, resume=snap)
    res = _drain(srv, 1)[1]
    srv.close()
    np.testing.assert_array_equal(res["popt"], ref["popt"])
    assert res["cost"] == ref["cost"] and res["nfev"] == ref["nfev"] and res["fit_status"] == ref["fit_status"]
    # a snapshot is refused for another size
    other = synth.dexp(30_001, seed=44, dtype=dtype)
    srv = gbfit.Server(hbm_budget_bytes=64 << 20, max_slots=4, precision=precision)
    with pytest.raises(gbfit.GbfitError) as e:
        _submit(srv, other, 2, resume=snap)
    assert e.value.code == gbfit.E_INVALID_ARG
    srv.close()
