"""GPU: tile shapes of the bulk-copy ring against the oracle.

Each CTA streams its tiles through a ring of four shared-memory stages that
the last warp to release a stage refills.  These tests run tile shapes that
take every path of that: tiles of fewer chunks than stages, of exactly and
of more than the stage count, a partial last chunk and a ragged last tile,
many tiles per CTA, with and without sigma, and check the sums against the
oracle's definition (mixed tolerance) and themselves across repeated
launches (bit for bit: the combine order is fixed by tile index, whatever
CTA ran a tile).
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


def dev(a):
    return None if a is None else torch.as_tensor(np.ascontiguousarray(a)).float().cuda()


@pytest.fixture(scope="module")
def prob():
    # about 4 to 30 tiles per CTA at the tile sizes below; ragged last tile
    return synth.gauss1d(4_000_000 + 1234, seed=31, with_sigma=True, dtype=np.float32)


@pytest.mark.parametrize("tile_points", [1024, 2048 * 3, 2048 * 4, 2048 * 4 + 512, 2048 * 9])
@pytest.mark.parametrize("with_sigma", [False, True])
def test_ring_tiles_match_definition_and_repeat(prob, tile_points, with_sigma):
    pr = prob
    sig = pr.sigma if with_sigma else None
    f, g, B, _, _ = red.evaluate(pr.model, pr.coords(), pr.y, red.weights(sig, pr.m), pr.p0)
    x, y, s = dev(pr.x), dev(pr.y), dev(sig)
    runs = [gbfit.evaluate(pr.model, x, y, pr.p0, sigma=s, precision="mixed", tile_points=tile_points)
            for _ in range(3)]
    for Bp, gg, cost in runs[1:]:
        np.testing.assert_array_equal(Bp, runs[0][0])
        np.testing.assert_array_equal(gg, runs[0][1])
        assert cost == runs[0][2]
    Bp, gg, cost = runs[0]
    Bg = gbfit.unpack_upper(Bp, pr.n)
    tol = 2e-5
    dscale = np.sqrt(np.outer(np.diag(B), np.diag(B)))
    assert np.max(np.abs(Bg - B) / dscale) <= tol
    assert np.max(np.abs(gg - g) / np.sqrt(np.diag(B) * 2 * f)) <= tol
    assert abs(cost - f) <= tol * f


def test_small_tile_fit_repeats_bitwise(prob):
    """A whole mixed fit over many small tiles per CTA: the same result on
    every launch, and within 1e-6 of the fit with the default tiles."""
    pr = prob
    x, y = dev(pr.x), dev(pr.y)
    tol = dict(ftol=1e-10, xtol=1e-10, gtol=1e-10)
    a = gbfit.curve_fit(pr.model, x, y, pr.p0, precision="mixed", tile_points=2048 * 4 + 512, **tol)
    b = gbfit.curve_fit(pr.model, x, y, pr.p0, precision="mixed", tile_points=2048 * 4 + 512, **tol)
    np.testing.assert_array_equal(a["popt"], b["popt"])
    assert a["nfev"] == b["nfev"] and a["cost"] == b["cost"]
    c = gbfit.curve_fit(pr.model, x, y, pr.p0, precision="mixed", **tol)
    assert np.max(np.abs(a["popt"] - c["popt"]) / np.maximum(np.abs(c["popt"]), 1.0)) <= 1e-6
