"""The allocation-free evaluation entry point (gbfit_evaluate_noalloc).

Some callers cannot allocate device memory when they call the library: an
application whose memory manager owns all device memory, or a loop that
cannot take the implicit device-wide synchronisation of cudaMalloc.
gbfit_evaluate_noalloc runs the same fused reduction pass as gbfit_evaluate
with its scratch in a fixed device array instead.  This checks, through the C
ABI, that two calls in a row return the same sums as gbfit_evaluate and as the
FP64 oracle's definition of the sums (the parity tests' tolerances: 1e-12 of
each entry's scale in plain FP64, 2e-5 in mixed precision), at an explicit and
at the default tile size, and that a request beyond the array's capacity is
refused.  The file name sorts last so that a run stopping at the first failure
has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import reduce as red
from paper_2208_12187_gb300 import build, gbfit, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return gbfit.load()


def _dev(a, dtype):
    return None if a is None else torch.as_tensor(np.ascontiguousarray(a)).to(dtype).cuda()


def _close(a, b, tol):
    Ba, ga, fa = a
    Bb, gb, fb = b
    scale = max(np.max(np.abs(Bb)), 1e-300)
    assert np.max(np.abs(Ba - Bb)) <= tol * scale
    assert np.max(np.abs(ga - gb)) <= tol * max(np.max(np.abs(gb)), np.sqrt(scale * fb), 1e-300)
    assert abs(fa - fb) <= tol * abs(fb)


def _close_oracle(out, pr, p, tol):
    """Sums against the oracle's definition (Eqs. msqe, gradient, hessian) at
    p, on the same data, scaled per entry as in the parity tests."""
    Bp, gg, cost = out
    f, g, B, _, _ = red.evaluate(pr.model, pr.coords(), pr.y, red.weights(pr.sigma, pr.m), p)
    Bg = gbfit.unpack_upper(Bp, pr.n)
    dscale = np.sqrt(np.outer(np.diag(B), np.diag(B)))
    assert np.max(np.abs(Bg - B) / np.maximum(dscale, 1e-300)) <= tol
    assert np.max(np.abs(gg - g) / np.maximum(np.sqrt(np.diag(B) * 2 * f), 1e-300)) <= tol
    assert abs(cost - f) <= tol * f


@pytest.mark.parametrize("tile_points", [2048, 0])
@pytest.mark.parametrize("precision,dtype,tol", [("fp64", torch.float64, 1e-12), ("mixed", torch.float32, 2e-5)])
def test_noalloc_matches_evaluate_and_oracle_twice(precision, dtype, tol, tile_points):
    cases = [synth.gauss1d(3 * 2048 + 17, seed=1, with_sigma=True),
             synth.gauss2d_grid(97, seed=4, dtype=np.float64)]
    for pr in cases:
        x = None if pr.layout == synth.LAYOUT_GRID else _dev(pr.x, dtype)
        y, s = _dev(pr.y, dtype), _dev(pr.sigma, dtype)
        kw = dict(sigma=s, grid_wh=pr.grid_wh, precision=precision, tile_points=tile_points)
        ref = gbfit.evaluate(pr.model, x, y, pr.p0, **kw)
        first = gbfit.evaluate_noalloc(pr.model, x, y, pr.p0, **kw)
        second = gbfit.evaluate_noalloc(pr.model, x, y, pr.p0, **kw)
        _close(first, ref, tol)
        _close(second, ref, tol)
        _close_oracle(first, pr, pr.p0, tol)
        _close_oracle(second, pr, pr.p0, tol)
        # a different parameter point through the same shared array
        p1 = pr.p0 * 1.01
        out1 = gbfit.evaluate_noalloc(pr.model, x, y, p1, **kw)
        _close(out1, gbfit.evaluate(pr.model, x, y, p1, **kw), tol)
        _close_oracle(out1, pr, p1, tol)


def test_noalloc_rejects_too_many_tiles():
    y = torch.zeros(2048 * 256 + 1, dtype=torch.float32, device="cuda")
    x = torch.zeros_like(y)
    with pytest.raises(gbfit.GbfitError) as e:
        gbfit.evaluate_noalloc(gbfit.MODEL_GAUSS1D, x, y, [1.0, 0.0, 1.0, 0.0], precision="mixed", tile_points=256)
    assert e.value.code == gbfit.E_INVALID_ARG
    assert "at most 2048 tiles" in str(e.value)
