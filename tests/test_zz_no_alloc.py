"""moses_step_static: the step for callers that cannot allocate device memory.

Callers that keep all device memory in their own pool, that run under a hard
device-memory limit, or whose loop may not stall on the allocator (cudaMalloc
synchronises the device) cannot let a library call cudaMalloc.
moses_step_static gives them one FP64 step with its scratch in a statically
sized device array.  These tests drive it through the C-ABI with device
buffers they own and check two calls in a row against the allocating path
(moses_create + moses_step) at the FP64 parity tolerance of the other GPU
tests, with closed and with transmissive sides, in place (output buffer = input
buffer), and that a non-finite input is reported.  They live in a file of their
own that pytest collects last.
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


@pytest.mark.parametrize("bc,in_place", [((0, 0, 0, 0), False), ((1, 1, 1, 1), False), ((0, 1, 1, 0), True)])
def test_static_step_matches_the_allocating_step_on_two_calls(bc, in_place):
    torch = pytest.importorskip("torch")
    L = moses.lib()
    nx, ny = 75, 61  # several 32 x 8 tiles with ragged tails, inside the 128 x 128 limit
    cfg = W.release_config(nx=nx, ny=ny, cfl=0.3)
    cfg["params"] = dict(cfg["params"], bc=bc)
    ref = moses.from_config(cfg)
    ref.step(40)  # the pile moving, so that the transmissive sides see flow
    dem_d = torch.tensor(cfg["dem"], dtype=torch.float64, device="cuda")
    Uin = torch.tensor(ref.get_conserved(), dtype=torch.float64, device="cuda")
    Uout = Uin if in_place else torch.empty_like(Uin)
    par = moses.Params.from_dict(cfg["params"])
    stream = torch.cuda.current_stream().cuda_stream
    t = ref.budget()["t"]
    for call in range(2):
        rc, dt = _call(L, dem_d, nx, ny, cfg["dx"], par, Uin, Uout, t, stream)
        assert rc == 0, L.moses_last_error(None).decode()
        t_ref = ref.step(1)
        err = _rel_maxnorm(Uout.cpu().numpy(), ref.get_conserved())
        assert err <= TOL64, f"call {call + 1}: static step departs from moses_step by {err}"
        assert abs((t + dt) - t_ref) <= 1e-12 * t_ref
        t += dt
        if not in_place:
            Uin.copy_(Uout)


def test_static_step_reports_a_non_finite_input():
    torch = pytest.importorskip("torch")
    L = moses.lib()
    nx, ny = 40, 24
    cfg = W.release_config(nx=nx, ny=ny, cfl=0.3)
    ref = moses.from_config(cfg)
    U = torch.tensor(ref.get_conserved(), dtype=torch.float64, device="cuda")
    U[1, ny // 2, nx // 2] = float("nan")
    dem_d = torch.tensor(cfg["dem"], dtype=torch.float64, device="cuda")
    par = moses.Params.from_dict(cfg["params"])
    rc, _ = _call(L, dem_d, nx, ny, cfg["dx"], par, U, torch.empty_like(U), 0.0, torch.cuda.current_stream().cuda_stream)
    assert rc == moses.MOSES_ENONFINITE
    assert b"non-finite" in L.moses_last_error(None)
    # the next call on a finite state succeeds: the shared scratch starts clean
    U2 = torch.tensor(ref.get_conserved(), dtype=torch.float64, device="cuda")
    out = torch.empty_like(U2)
    rc, _ = _call(L, dem_d, nx, ny, cfg["dx"], par, U2, out, 0.0, torch.cuda.current_stream().cuda_stream)
    assert rc == 0, L.moses_last_error(None).decode()
    ref.step(1)
    assert _rel_maxnorm(out.cpu().numpy(), ref.get_conserved()) <= TOL64


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
