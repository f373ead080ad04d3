"""moses_step_static: the step for callers that cannot allocate device memory.

Callers that record their work into a CUDA graph, that keep all device memory
in their own pool, or that run under a hard device-memory limit cannot let a
library call cudaMalloc.  moses_step_static gives them one FP64 step with its
scratch in a statically sized device array.  This test drives it through the
C-ABI with device buffers it owns and checks two calls in a row against the
allocating path (moses_create + moses_step) at the FP64 parity tolerance of the
other GPU tests.  It lives in a file of its own that pytest collects last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2104_06784_gb300 import moses, workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def _rel_maxnorm(a, b):
    scale = np.abs(b).reshape(6, -1).max(axis=1)
    scale = np.where(scale > 0, scale, 1.0)
    return float((np.abs(a - b).reshape(6, -1).max(axis=1) / scale).max())


def _call(L, dem_d, nx, ny, dx, par, Uin, Uout, t, stream):
    dt = C.c_double()
    rc = L.moses_step_static(C.c_void_p(dem_d.data_ptr()), nx, ny, dx, dx, C.byref(par), C.c_void_p(Uin.data_ptr()),
                             C.c_void_p(Uout.data_ptr()), t, C.byref(dt), C.c_void_p(stream))
    return rc, dt.value


def test_static_step_matches_the_allocating_step_on_two_calls():
    torch = pytest.importorskip("torch")
    L = moses.lib()
    nx, ny = 75, 61  # several 32 x 8 tiles with ragged tails, inside the 128 x 128 limit
    cfg = W.release_config(nx=nx, ny=ny, cfl=0.3)
    ref = moses.from_config(cfg)
    dem_d = torch.tensor(cfg["dem"], dtype=torch.float64, device="cuda")
    Uin = torch.tensor(ref.get_conserved(), dtype=torch.float64, device="cuda")
    Uout = torch.empty_like(Uin)
    par = moses.Params.from_dict(cfg["params"])
    stream = torch.cuda.current_stream().cuda_stream
    t = 0.0
    for call in range(2):
        rc, dt = _call(L, dem_d, nx, ny, cfg["dx"], par, Uin, Uout, t, stream)
        assert rc == 0, L.moses_last_error(None).decode()
        t_ref = ref.step(1)
        err = _rel_maxnorm(Uout.cpu().numpy(), ref.get_conserved())
        assert err <= TOL64, f"call {call + 1}: static step departs from moses_step by {err}"
        assert abs((t + dt) - t_ref) <= 1e-12 * t_ref
        t += dt
        Uin.copy_(Uout)


def test_static_step_rejects_grids_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    L = moses.lib()
    nx, ny = 129, 8
    dem_d = torch.zeros((ny, nx), dtype=torch.float64, device="cuda")
    U = torch.zeros((6, ny, nx), dtype=torch.float64, device="cuda")
    par = moses.Params.from_dict(W.default_params())
    rc, _ = _call(L, dem_d, nx, ny, 5.0, par, U, U, 0.0, torch.cuda.current_stream().cuda_stream)
    assert rc == moses.MOSES_EINVAL
    assert b"128" in L.moses_last_error(None)
