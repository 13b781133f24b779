"""The trust-region step's FP64 reciprocal (rcp64: Newton-Raphson from the
correctly rounded FP32 reciprocal), through gbfit_check_rcp64, against the
correctly rounded 1.0 / x: within 1 ulp of the result on [1e-36, 1e36] in
magnitude (log-uniform, both signs, powers of two and the range's edges), and
exactly the division outside that range (its fallback)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2208_12187_gb300 import build, gbfit

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return gbfit.load()


def test_rcp64_within_one_ulp_on_its_range():
    rng = np.random.default_rng(0)
    mag = 10.0 ** rng.uniform(-36.0, 36.0, 400_000)
    x = mag * rng.choice([-1.0, 1.0], mag.size)
    edges = np.array([1e-36 * (1 + 1e-9), 1e36 * (1 - 1e-9), 1.0, -1.0, 3.0, 1.0 / 3.0, np.pi, 0.1])
    pow2 = np.ldexp(1.0, np.arange(-119, 120))
    x = np.concatenate([x, edges, pow2, -pow2, np.nextafter(pow2, 0), np.nextafter(pow2, 2 * pow2)])
    x = x[(np.abs(x) > 1e-36) & (np.abs(x) < 1e36)]
    y = gbfit.check_rcp64(torch.as_tensor(x).cuda()).cpu().numpy()
    ref = 1.0 / x
    ulp = np.abs(y - ref) / np.spacing(np.abs(ref))
    assert ulp.max() <= 1.0, (x[np.argmax(ulp)], ulp.max())
    assert np.mean(ulp == 0.0) >= 0.9            # mostly the correctly rounded result


def test_rcp64_outside_its_range_is_the_division():
    x = np.array([1e-300, -1e-300, 1e-37, 1e37, 1e300, -1e300, 5e-324, np.inf, -np.inf, 1e-36, 1e36])
    y = gbfit.check_rcp64(torch.as_tensor(x).cuda()).cpu().numpy()
    with np.errstate(divide="ignore", over="ignore"):
        ref = 1.0 / x
    np.testing.assert_array_equal(y, ref)
