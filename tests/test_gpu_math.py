"""The stage kernels' own reciprocal and square roots against CUDA's results
and against the exact values.

The FP64 form of the stage kernel does not call CUDA's division or square
root: it starts from the hardware approximations (rcp.approx / rsqrt.approx,
relative error about 2^-23) and takes one third-order refinement step each,
from the series (1 - e)^-1 = 1 + e + e^2 + ... for the reciprocal (e = 1 - x y,
Newton-Raphson's iteration for 1/x carried to third order, as in
Markstein's analysis of division by iterative refinement) and
(1 - d)^-1/2 = 1 + d/2 + 3 d^2/8 + ... for the square roots (d = 1 - x y^2,
the third-order Householder step for 1/sqrt(x)).  Each step cubes the
relative error, so from 2^-23 it lands within an ulp of the exact result.
These tests run the functions on the GPU (moses_debug_math) over
logarithmically spaced inputs and random mantissas across the exponent range,
subnormals included where the function is defined for them, and hold each to
its bound in ulps of the exact value, and to within an ulp or two of CUDA's
own 1.0/x, sqrt and rsqrt.
"""
import numpy as np
import pytest

from paper_2104_06784_gb300 import moses

pytestmark = pytest.mark.gpu

# bounds in ulps of the exact result (the measured maxima stay below them)
BOUND = {"frcp": 1.0, "fsqrt": 0.76, "frsqrt": 0.99}


def _inputs(lo_exp, hi_exp, n=200_000, seed=0):
    rng = np.random.default_rng(seed)
    x = np.logspace(lo_exp, hi_exp, n // 2)
    m = rng.uniform(1.0, 2.0, n // 2)
    k = rng.integers(int(lo_exp * 3.3219), int(hi_exp * 3.3219), n // 2)
    return np.concatenate([x, np.ldexp(m, k)])


def _ulps(f, exact):
    """|f - exact| in ulps of the exact value rounded to FP64 (exact as long double)."""
    e64 = exact.astype(np.float64)
    return (np.abs(f.astype(np.longdouble) - exact) / np.spacing(np.abs(e64)).astype(np.longdouble)).astype(np.float64)


def test_fp64_reciprocal_within_an_ulp():
    # defined where both x and 1/x are normal numbers
    x = _inputs(-307.0, 307.0)
    r = moses.debug_math(x)
    exact = np.longdouble(1) / x.astype(np.longdouble)
    u = _ulps(r["frcp"], exact)
    assert u.max() <= BOUND["frcp"], f"frcp: {u.max():.3f} ulp at x = {x[u.argmax()]!r}"
    # CUDA's 1.0/x is correctly rounded: the two agree to an ulp
    assert np.all(np.abs(r["frcp"] - r["cuda_rcp"]) <= np.spacing(np.abs(r["cuda_rcp"])))


def test_fp64_square_root_within_its_bound_and_zero_below_normal():
    x = _inputs(-307.0, 307.0)
    r = moses.debug_math(x)
    exact = np.sqrt(x.astype(np.longdouble))
    u = _ulps(r["fsqrt"], exact)
    assert u.max() <= BOUND["fsqrt"], f"fsqrt: {u.max():.3f} ulp at x = {x[u.argmax()]!r}"
    assert np.all(np.abs(r["fsqrt"] - r["cuda_sqrt"]) <= np.spacing(r["cuda_sqrt"]))
    # documented: 0 for x <= 0 and for subnormal x (the dry cells' speeds)
    sub = np.array([0.0, -0.0, -1.0, 5e-324, 1e-310, 2.2e-308])
    assert np.all(moses.debug_math(sub)["fsqrt"] == 0.0)


def test_fp64_reciprocal_square_root_within_its_bound_subnormals_included():
    x = np.concatenate([_inputs(-307.0, 307.0, seed=1), np.logspace(-323, -307.7, 2000)])
    r = moses.debug_math(x)
    exact = np.longdouble(1) / np.sqrt(x.astype(np.longdouble))
    u = _ulps(r["frsqrt"], exact)
    assert u.max() <= BOUND["frsqrt"], f"frsqrt: {u.max():.3f} ulp at x = {x[u.argmax()]!r}"
    assert np.all(np.abs(r["frsqrt"] - r["cuda_rsqrt"]) <= 2 * np.spacing(np.abs(r["cuda_rsqrt"])))


def test_fp32_forms_within_two_ulps():
    # the FP32 form uses the hardware approximations unrefined
    x = _inputs(-37.5, 37.5, seed=2).astype(np.float32).astype(np.float64)
    r = moses.debug_math(x)
    xf = x.astype(np.float32).astype(np.longdouble)
    for name, exact in (("frcp32", np.longdouble(1) / xf), ("fsqrt32", np.sqrt(xf)),
                        ("frsqrt32", np.longdouble(1) / np.sqrt(xf))):
        e32 = exact.astype(np.float32)
        u = (np.abs(r[name].astype(np.longdouble) - exact)
             / np.spacing(np.abs(e32)).astype(np.longdouble)).astype(np.float64)
        assert u.max() <= 2.0, f"{name}: {u.max():.3f} ulp at x = {x[u.argmax()]!r}"
