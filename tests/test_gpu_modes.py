"""The loop kernel's two hand-off modes give bitwise-identical fits.

A launch of at most 8 fits runs each fit's final combine and trust-region
step in a fixed owner CTA; a larger launch gives them to the last arriving
group.  Both sum the group partials in index order and run the same step, so
a fit's results must not depend on the mode (nor on the other fits).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2208_12187_gb300 import build, gbfit, synth

pytestmark = pytest.mark.gpu
TOL = dict(ftol=1e-10, xtol=1e-10, gtol=1e-10)


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return gbfit.load()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_owner_and_last_arriver_modes_agree(precision):
    dt = np.float32 if precision == "mixed" else np.float64
    tdt = torch.float32 if precision == "mixed" else torch.float64
    rng = np.random.default_rng(5)
    # sizes spanning one and several combine groups (tiles of 2048 points, 4 tiles a group);
    # multiples of 4 points, so that every fit's data starts 16-byte aligned in the
    # concatenated batch as it does alone (the mixed path's bulk copies split a
    # tile at the first 16-byte boundary, which sets the point-to-thread mapping)
    sizes = [4 * int(v) for v in rng.integers(750, 37_500, 9)]
    probs = [synth.gauss1d(m, seed=40 + k).astype(dt) for k, m in enumerate(sizes)]
    kw = dict(precision=precision, tile_points=2048, group_tiles=4, **TOL)

    def batch(ps):
        off = np.concatenate([[0], np.cumsum([p.m for p in ps])]).astype(np.int64)
        x = torch.as_tensor(np.concatenate([p.x for p in ps])).to(tdt).cuda()
        y = torch.as_tensor(np.concatenate([p.y for p in ps])).to(tdt).cuda()
        return gbfit.curve_fit_batch(0, off, x, y, np.stack([p.p0 for p in ps]), **kw)

    alone = [gbfit.curve_fit(0, torch.as_tensor(p.x).cuda(), torch.as_tensor(p.y).cuda(), p.p0, **kw) for p in probs]
    eight = batch(probs[:8])          # owner mode
    nine = batch(probs)               # last-arriver mode
    for k, a in enumerate(alone):
        np.testing.assert_array_equal(nine["popt"][k], a["popt"])
        assert nine["cost"][k] == a["cost"] and nine["nfev"][k] == a["nfev"]
        if k < 8:
            np.testing.assert_array_equal(eight["popt"][k], a["popt"])
            assert eight["cost"][k] == a["cost"] and eight["nfev"][k] == a["nfev"]
