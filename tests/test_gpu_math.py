"""The library's own FP64 reciprocal and reciprocal square root (Newton
steps from FP32 seeds, used on the dependent chains of the dense reduced
algebra) held against CUDA's correctly rounded FP64 division and its
square root, over random and edge inputs, including those outside the FP32
range that take the FP64 fallback."""
import numpy as np
import pytest

from paper_2301_01718_gb300 import hyrom as H
from tests.gpu_util import torch

pytestmark = pytest.mark.gpu


def _inputs(positive):
    g = np.random.Generator(np.random.PCG64(11))
    x = np.exp(g.uniform(np.log(1e-36), np.log(1e36), 200000))
    x *= 1.0 + g.uniform(-1e-3, 1e-3, x.size)       # mantissas off the FP32 grid
    edge = np.array([1.0, 2.0, 3.0, 0.5, 0.1, 1.0 / 3.0, 7.0, 1e-300, 1e300, 5e-324,
                     2.2250738585072014e-308, 1.17549435e-38, 1.1754943e-38, 1.17549436e-38,
                     1.7e38, 1.69999e38, 1.70001e38, 3.4e38, 1e-45, 1e308,
                     np.nextafter(1.0, 2.0), np.nextafter(1.0, 0.0)])
    x = np.concatenate([x, edge])
    if not positive:
        x = np.concatenate([x, -x])
    return x


def _run(which, x):
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    yd = torch.empty_like(xd)
    H.hyrom_selftest_math(which, xd, yd)
    torch.cuda.synchronize()
    return xd, yd


def test_reciprocal_within_two_ulp_of_division():
    x = _inputs(positive=False)
    xd, yd = _run(0, x)
    ref = (1.0 / xd).cpu().numpy()
    y = yd.cpu().numpy()
    fin = np.isfinite(ref) & (ref != 0)
    ulp = np.abs(y[fin] - ref[fin]) / np.spacing(np.abs(ref[fin]))
    assert ulp.max() <= 2.0, ulp.max()
    assert np.array_equal(y[~fin], ref[~fin])
    # the FP64 fallback outside the FP32 range is the division itself
    out = np.abs(x) > 1.7e38
    assert np.array_equal(y[out], ref[out])


def test_reciprocal_square_root_within_three_ulp():
    x = _inputs(positive=True)
    xd, yd = _run(1, x)
    ref = (1.0 / torch.sqrt(xd)).cpu().numpy()   # two correctly rounded steps: < 1.5 ulp
    y = yd.cpu().numpy()
    fin = np.isfinite(ref)
    ulp = np.abs(y[fin] - ref[fin]) / np.spacing(ref[fin])
    assert ulp.max() <= 3.0, ulp.max()
    # a property of the exact value: x y^2 = 1 within a few ulp
    mid = (x > 1e-300) & (x < 1e300)
    r = x[mid] * y[mid] * y[mid]
    assert np.abs(r - 1.0).max() < 8 * np.finfo(np.float64).eps


def test_selftest_rejects_bad_arguments():
    xd = torch.ones(4, dtype=torch.float64, device="cuda")
    with pytest.raises(H.HyromError):
        H.hyrom_selftest_math(2, xd, xd.clone())
