"""The kernels replace the IEEE FP64 division 1/h, square root sqrt(g h) and
reciprocal square root by their own routines (FP32 seed from the bit
pattern, one third-order refinement).  Their error against the correctly
rounded result must stay within one ulp over the range the path uses and
far beyond it."""
import numpy as np
import pytest

from gpu_common import load, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def crk():
    return load()


def ulps(got, want):
    return np.abs(got - want) / np.spacing(np.abs(want))


def samples():
    rng = np.random.default_rng(5)
    a = np.exp(rng.uniform(np.log(1e-30), np.log(1e30), 200000))
    b = rng.uniform(0.05, 3.0, 200000)               # depths of the workloads
    c = np.array([1.0, 2.0, 0.5, 0.1, 9.81, 1e-300, 1e300, 3.0e38, 1.1e-38])
    return np.concatenate([a, b, c])


def test_reciprocal_within_one_ulp(crk):
    x = samples()
    x = np.concatenate([x, -x])
    got = to_host(crk.math_check(to_dev(x), "rcp"))
    assert np.max(ulps(got, 1.0 / x)) <= 1.0


def test_sqrt_within_one_ulp(crk):
    x = samples()
    got = to_host(crk.math_check(to_dev(x), "sqrt"))
    assert np.max(ulps(got, np.sqrt(x))) <= 1.0


def test_rsqrt_within_one_ulp(crk):
    """1/sqrt(x) (the shallow-water wave speed and the time-step rate use it)
    against the reciprocal square root in extended precision, rounded once."""
    x = samples()
    got = to_host(crk.math_check(to_dev(x), "rsqrt"))
    ref = (1.0 / np.sqrt(x.astype(np.longdouble))).astype(np.float64)
    assert np.max(ulps(got, ref)) <= 1.0


def test_fp64_probe_rates_are_plausible():
    """The FP64 throughput probe returns finite rates below the unit-count
    peak of any sm_103 part (152 SMs x 2 FMA/clk x 2 flop x 2.1 GHz) and
    well above zero, for each mode."""
    from gpu_common import load
    crk = load()
    for mode in ("fma", "mma", "both"):
        t = crk.fp64_probe(mode, blocks=304, iters=1024, repeats=2)
        assert 0.05 < t < 1.4, (mode, t)
