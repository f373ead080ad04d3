"""The C-ABI library loads and exports every entry point of include/*.h.

CPU only: no call here touches a GPU (argument validation returns before any
CUDA call).
"""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

from paper_2104_06784_gb300 import build as B
from paper_2104_06784_gb300 import moses, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return moses.lib()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(moses_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), f"{n} declared in include/ but not exported"


def test_binding_covers_the_header():
    bound = {n for n, _, _ in moses.SIGNATURES}
    assert set(_declared()) <= bound


def test_version(L):
    assert b"sm_103a" in L.moses_version()


def _create(dem, nx, ny, dx=5.0, dy=5.0, **over):
    p = moses.Params.from_dict(W.default_params(**over))
    h = C.c_void_p()
    d = np.ascontiguousarray(dem, dtype=np.float64)
    rc = moses.lib().moses_create(d.ctypes.data_as(C.POINTER(C.c_double)), nx, ny, dx, dy, C.byref(p), None,
                                  C.byref(h))
    return rc, h


@pytest.mark.parametrize("nx,ny,dx,over", [
    (0, 4, 5.0, {}), (4, 0, 5.0, {}), (4, 4, 0.0, {}), (4, 4, -1.0, {}), (4, 4, float("nan"), {}),
    (4, 4, 5.0, dict(cfl=0.0)), (4, 4, 5.0, dict(rho_f=3000.0)), (4, 4, 5.0, dict(h_dry=0.0)),
    (4, 4, 5.0, dict(bc=(0, 2, 0, 0))), (4, 4, 5.0, dict(k_mode=2)), (4, 4, 5.0, dict(k_mode=1, phi_int_deg=20.0)), (4, 4, 5.0, dict(k_mode=1, scheme=1)), (4, 4, 5.0, dict(delta_b_deg=95.0)),
    (4, 4, 5.0, dict(c_d=-1.0)), (4, 4, 5.0, dict(g=0.0)), (4, 4, 5.0, dict(fluid_pg_mode=3)),
])
def test_create_rejects_bad_arguments(L, nx, ny, dx, over):
    rc, h = _create(np.zeros((max(ny, 1), max(nx, 1))), nx, ny, dx, dx, **over)
    assert rc == moses.MOSES_EINVAL
    assert not h.value
    assert L.moses_last_error(None)


def test_create_rejects_nonfinite_dem(L):
    dem = np.zeros((3, 3))
    dem[1, 1] = np.inf
    rc, h = _create(dem, 3, 3)
    assert rc == moses.MOSES_EINVAL and b"non-finite" in L.moses_last_error(None)


def test_null_pointers(L):
    assert L.moses_create(None, 4, 4, 1.0, 1.0, None, None, None) == moses.MOSES_EINVAL
    assert L.moses_step(None, 1, None) == moses.MOSES_EINVAL
    L.moses_destroy(None)


@pytest.mark.parametrize("field,value", [("scheme", 2), ("recon", 2), ("recon", -1), ("rk", 1), ("rk", 4)])
def test_create_rejects_bad_scheme_options(L, field, value):
    rc, h = _create(np.zeros((4, 4)), 4, 4, **{field: value})
    assert rc == moses.MOSES_EINVAL and field.encode() in L.moses_last_error(None)
