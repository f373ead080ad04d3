"""Python binding of the C-ABI in include/moses.h (argument marshalling only).

Every computation of the step runs in the CUDA kernels of libmoses.so; this
module only converts arguments and return codes.  There is no CPU fallback:
if the library has not been built, or cannot find a GPU, calls fail with
``MosesError``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmoses.so")

MOSES_OK, MOSES_EINVAL, MOSES_ENOMEM, MOSES_ECUDA, MOSES_ENONFINITE, MOSES_ETIMEOUT, MOSES_ESTATE = 0, -1, -2, -3, -4, -5, -6
FP64, FP32 = 0, 1
BUDGET_LEN = 13
BUDGET_KEYS = ("vol_s", "vol_f", "mom_xs", "mom_ys", "mom_xf", "mom_yf", "bnd_in_s", "bnd_in_f",
               "clamp_s", "clamp_f", "clamp_cells", "t", "steps")


class MosesError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"moses error {code}: {msg}")
        self.code = code


class Params(C.Structure):
    """moses_params of include/moses.h."""
    _fields_ = [("g", C.c_double), ("eps", C.c_double), ("eps_chi", C.c_double),
                ("rho_s", C.c_double), ("rho_f", C.c_double),
                ("delta_b_deg", C.c_double), ("phi_int_deg", C.c_double), ("k_mode", C.c_int),
                ("c_d", C.c_double), ("nu_f", C.c_double), ("k_f", C.c_double),
                ("cfl", C.c_double), ("dt_max", C.c_double), ("h_dry", C.c_double),
                ("bc", C.c_int * 4), ("fluid_pg_mode", C.c_int), ("precision", C.c_int), ("scheme", C.c_int),
                ("recon", C.c_int), ("rk", C.c_int)]

    @classmethod
    def from_dict(cls, p: dict, precision: int = FP64) -> "Params":
        s = cls()
        for name, _ in cls._fields_:
            if name == "bc":
                s.bc[:] = [int(v) for v in p["bc"]]
            elif name in ("k_mode", "fluid_pg_mode"):
                setattr(s, name, int(p[name]))
            elif name == "precision":
                s.precision = int(p.get("precision", precision))
            elif name in ("scheme", "recon", "rk"):
                setattr(s, name, int(p.get(name, 2 if name == "rk" else 0)))
            else:
                setattr(s, name, float(p[name]))
        return s


_lib = None
_dp = C.POINTER(C.c_double)
_vp = C.c_void_p

# (name, restype, argtypes) of every entry point declared in include/moses.h
SIGNATURES = [
    ("moses_create", C.c_int, [_dp, C.c_int, C.c_int, C.c_double, C.c_double, C.POINTER(Params), _vp,
                               C.POINTER(_vp)]),
    ("moses_set_release", C.c_int, [_vp, _dp, _dp, _dp, _dp, _dp, _dp]),
    ("moses_set_inflow", C.c_int, [_vp, C.c_int, C.c_int, C.c_int, C.c_int, _dp, _dp, _dp]),
    ("moses_step", C.c_int, [_vp, C.c_int, _dp]),
    ("moses_step_timed", C.c_int, [_vp, C.c_int, _dp, _dp]),
    ("moses_step_dt", C.c_int, [_vp, C.c_int, C.c_double, _dp]),
    ("moses_set_tile", C.c_int, [_vp, C.c_int]),
    ("moses_autotune", C.c_int, [_vp, C.c_int, C.POINTER(C.c_int), _dp]),
    ("moses_run_until", C.c_int, [_vp, C.c_double, C.c_int, C.POINTER(C.c_int)]),
    ("moses_next_dt", C.c_int, [_vp, _dp, _dp]),
    ("moses_get_state", C.c_int, [_vp, _dp, _dp, _dp, _dp, _dp, _dp]),
    ("moses_get_conserved", C.c_int, [_vp, _dp]),
    ("moses_set_conserved", C.c_int, [_vp, _dp]),
    ("moses_get_conserved_device", C.c_int, [_vp, _vp]),
    ("moses_set_conserved_device", C.c_int, [_vp, _vp]),
    ("moses_stage", C.c_int, [_vp, C.c_double, C.c_double, _dp]),
    ("moses_max_speed", C.c_int, [_vp, _dp]),
    ("moses_set_owned_rows", C.c_int, [_vp, C.c_int, C.c_int]),
    ("moses_row_planes", C.c_int, [_vp]),
    ("moses_get_rows_device", C.c_int, [_vp, C.c_int, C.c_int, _vp]),
    ("moses_set_rows_device", C.c_int, [_vp, C.c_int, C.c_int, _vp]),
    ("moses_set_max_speed", C.c_int, [_vp, C.c_double]),
    ("moses_get_budget", C.c_int, [_vp, _dp]),
    ("moses_step_static", C.c_int, [_vp, C.c_int, C.c_int, C.c_double, C.c_double, C.POINTER(Params), _vp, _vp,
                                    C.c_double, _dp, _vp]),
    ("moses_batch_create", C.c_int, [C.c_int, C.POINTER(_vp), C.POINTER(_vp)]),
    ("moses_batch_step", C.c_int, [_vp, C.c_int]),
    ("moses_batch_step_timed", C.c_int, [_vp, C.c_int, _dp]),
    ("moses_batch_tiles", C.c_int, [_vp]),
    ("moses_batch_tile_rows", C.c_int, [_vp, _dp]),
    ("moses_batch_set_tile_rows", C.c_int, [_vp, C.c_int]),
    ("moses_batch_debug_timeout", C.c_int, [_vp, C.c_int]),
    ("moses_batch_last_error", C.c_char_p, [_vp]),
    ("moses_batch_destroy", None, [_vp]),
    ("moses_adjoint_misfit", C.c_int, [_vp, C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp]),
    ("moses_stage_adjoint", C.c_int, [_vp, C.c_double, C.c_double, _dp, _dp, _dp]),
    ("moses_last_error", C.c_char_p, [_vp]),
    ("moses_destroy", None, [_vp]),
    ("moses_version", C.c_char_p, []),
    ("moses_debug_timeout", C.c_int, [_vp, C.c_int]),
    ("moses_debug_poison", C.c_int, [_vp]),
    ("moses_debug_math", C.c_int, [_dp, C.c_int, _dp]),
    ("moses_debug_fp64_rate", C.c_int, [C.c_int, _dp]),
    ("moses_debug_flux_eval", C.c_int, [C.c_longlong, C.c_int, _dp]),
]


def lib():
    """Load libmoses.so; raise if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise MosesError(MOSES_ECUDA, f"{LIB_PATH} is missing: build it with "
                                          "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _f64(a):
    if a is None:
        return None
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


class Sim:
    """One simulation on the GPU (moses_create .. moses_destroy)."""

    def __init__(self, dem, dx: float, dy: float, params: dict, precision: int = FP64, stream=None):
        L = lib()
        self._L = L
        self.dem = _f64(dem)
        self.ny, self.nx = self.dem.shape
        self.dx, self.dy = float(dx), float(dy)
        self.params = dict(params)
        self.precision = int(params.get("precision", precision))
        self._par = Params.from_dict(params, self.precision)
        self._stream = _stream_ptr(stream)
        h = C.c_void_p()
        rc = L.moses_create(_p(self.dem), self.nx, self.ny, self.dx, self.dy, C.byref(self._par), self._stream,
                            C.byref(h))
        if rc != 0:
            raise MosesError(rc, L.moses_last_error(None).decode())
        self._h = h

    def _ck(self, rc):
        if rc != 0:
            raise MosesError(rc, self._L.moses_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._L.moses_destroy(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # inputs -----------------------------------------------------------------
    def set_release(self, h, phi_s=None, vx_s=None, vy_s=None, vx_f=None, vy_f=None):
        arrs = [_f64(a) for a in (h, phi_s, vx_s, vy_s, vx_f, vy_f)]
        self._ck(self._L.moses_set_release(self._h, *[_p(a) for a in arrs]))

    def set_inflow(self, side: int, i0: int, i1: int, t, Q, phi):
        t, Q, phi = _f64(t), _f64(Q), _f64(phi)
        self._ck(self._L.moses_set_inflow(self._h, side, i0, i1, len(t), _p(t), _p(Q), _p(phi)))

    def set_conserved(self, U):
        U = _f64(U)
        assert U.shape == (6, self.ny, self.nx)
        self._ck(self._L.moses_set_conserved(self._h, _p(U)))

    def set_conserved_device(self, ptr: int):
        self._ck(self._L.moses_set_conserved_device(self._h, C.c_void_p(ptr)))

    # stepping ---------------------------------------------------------------
    def step(self, n: int = 1) -> float:
        t = C.c_double()
        self._ck(self._L.moses_step(self._h, int(n), C.byref(t)))
        return t.value

    def step_timed(self, n: int = 1):
        """Advance n steps; returns (t, [stage-1 ms, stage-2 ms]) summed over
        the launches, measured with CUDA events on the simulation's stream."""
        t = C.c_double()
        ms = (C.c_double * 2)()
        self._ck(self._L.moses_step_timed(self._h, int(n), C.byref(t), ms))
        return t.value, [ms[0], ms[1]]

    def debug_timeout(self, on: bool = True):
        """Make the classification's bounded copy wait run out (testing the
        MOSES_ETIMEOUT path without a fault); False restores normal steps."""
        self._ck(self._L.moses_debug_timeout(self._h, int(bool(on))))

    def debug_poison(self):
        """Fill the never-read pitch padding of the device buffers with NaN."""
        self._ck(self._L.moses_debug_poison(self._h))

    # tile shape of the stage kernel -------------------------------------------
    TILES = {0: "32x8", 1: "32x4", 2: "32x16", 3: "32x4-2t"}  # 32x4-2t: two threads per cell
    TILE_SHAPES = {0: (32, 8), 1: (32, 4), 2: (32, 16), 3: (32, 4)}  # cells of each tile

    def set_tile(self, tile: int):
        self._ck(self._L.moses_set_tile(self._h, int(tile)))
        self._tile = int(tile)

    def tile_name(self) -> str:
        """The tile shape the stepping launches use (set_tile / autotune; 32x8 by default)."""
        return self.TILES[getattr(self, "_tile", 0)]

    def autotune(self, reps: int = 5, timings: bool = True):
        """Time one stage with each tile shape, keep the fastest; returns
        (tile, [ms per launch for each tile]) (timings: None when the cached
        choice was taken with timings=False)."""
        t = C.c_int()
        ms = np.zeros(len(self.TILES)) if timings else None
        self._ck(self._L.moses_autotune(self._h, int(reps), C.byref(t), _p(ms)))
        self._tile = t.value
        return t.value, (None if ms is None else [float(x) for x in ms])

    def step_dt(self, dt: float, n: int = 1) -> float:
        t = C.c_double()
        self._ck(self._L.moses_step_dt(self._h, int(n), float(dt), C.byref(t)))
        return t.value

    def run_until(self, t_end: float, max_steps: int = 10 ** 9) -> int:
        n = C.c_int()
        self._ck(self._L.moses_run_until(self._h, float(t_end), int(max_steps), C.byref(n)))
        return n.value

    def next_dt(self):
        dt, t = C.c_double(), C.c_double()
        self._ck(self._L.moses_next_dt(self._h, C.byref(dt), C.byref(t)))
        return dt.value, t.value

    def stage(self, t: float, dt: float) -> np.ndarray:
        out = np.empty((6, self.ny, self.nx))
        self._ck(self._L.moses_stage(self._h, float(t), float(dt), _p(out)))
        return out

    # outputs ----------------------------------------------------------------
    def max_speed(self) -> float:
        a = C.c_double()
        self._ck(self._L.moses_max_speed(self._h, C.byref(a)))
        return a.value

    def get_conserved(self, out=None) -> np.ndarray:
        U = np.empty((6, self.ny, self.nx)) if out is None else out
        self._ck(self._L.moses_get_conserved(self._h, _p(U)))
        return U

    def get_conserved_device(self, ptr: int):
        self._ck(self._L.moses_get_conserved_device(self._h, C.c_void_p(ptr)))

    # one strip of a row-decomposed domain (decomp.py) -------------------------
    def set_owned_rows(self, j0: int, j1: int):
        self._ck(self._L.moses_set_owned_rows(self._h, int(j0), int(j1)))

    @property
    def row_planes(self) -> int:
        return int(self._L.moses_row_planes(self._h))

    def get_rows_device(self, j0: int, nrows: int, ptr: int):
        """Rows [j0, j0 + nrows) into the device buffer at ptr
        (row_planes x nrows x nx doubles), asynchronous on the stream."""
        self._ck(self._L.moses_get_rows_device(self._h, int(j0), int(nrows), C.c_void_p(ptr)))

    def set_rows_device(self, j0: int, nrows: int, ptr: int):
        self._ck(self._L.moses_set_rows_device(self._h, int(j0), int(nrows), C.c_void_p(ptr)))

    def set_max_speed(self, amax: float):
        self._ck(self._L.moses_set_max_speed(self._h, float(amax)))

    def get_state(self) -> dict:
        arrs = [np.empty((self.ny, self.nx)) for _ in range(6)]
        self._ck(self._L.moses_get_state(self._h, *[_p(a) for a in arrs]))
        return dict(zip(("h", "phi_s", "vx_s", "vy_s", "vx_f", "vy_f"), arrs))

    def stage_adjoint(self, t: float, dt: float, lam_out):
        """(dS/dU)^T lam_out for one stage at the current state; also the
        parameter partials [d/d tan(delta_b), d/d c_D, d/d phi_int (per radian)]."""
        lo = _f64(lam_out)
        li = np.empty((6, self.ny, self.nx))
        gp = np.zeros(3)
        self._ck(self._L.moses_stage_adjoint(self._h, float(t), float(dt), _p(lo), _p(li), _p(gp)))
        return li, gp

    def adjoint_misfit(self, nsteps: int, hs_target, ckpt_every: int = 0, release_phi=None,
                       want_state=False, want_release=True):
        """Loss, parameter gradients [d/d delta_b (per deg), d/d phi_int, d/d c_D],
        dL/dh of the release and optionally dL/dU at the start; timings [ms]."""
        tgt = _f64(hs_target)
        loss = C.c_double()
        gp = np.zeros(3)
        gs = np.empty((6, self.ny, self.nx)) if want_state else None
        gh = np.empty((self.ny, self.nx)) if want_release else None
        phi = _f64(release_phi)
        tm = np.zeros(2)
        self._ck(self._L.moses_adjoint_misfit(self._h, int(nsteps), int(ckpt_every), _p(tgt), C.byref(loss), _p(gp),
                                              _p(gs), _p(gh), _p(phi), _p(tm)))
        return dict(loss=loss.value, g_params=gp, g_state0=gs, g_release_h=gh, timing_ms=tm)

    def budget(self) -> dict:
        out = np.empty(BUDGET_LEN)
        self._ck(self._L.moses_get_budget(self._h, _p(out)))
        return dict(zip(BUDGET_KEYS, out.tolist()))


class Batch:
    """An ensemble of simulations advanced together (moses_batch_*)."""

    def __init__(self, sims):
        self._L = lib()
        self.sims = list(sims)
        arr = (_vp * len(self.sims))(*[s._h.value for s in self.sims])
        h = C.c_void_p()
        rc = self._L.moses_batch_create(len(self.sims), arr, C.byref(h))
        if rc != 0:
            raise MosesError(rc, self._L.moses_batch_last_error(None).decode())
        self._h = h

    def step(self, n: int = 1):
        rc = self._L.moses_batch_step(self._h, int(n))
        if rc != 0:
            raise MosesError(rc, self._L.moses_batch_last_error(self._h).decode())

    def step_timed(self, n: int = 1) -> float:
        """Advance n steps; device time [ms] from CUDA events on the batch stream."""
        ms = C.c_double()
        rc = self._L.moses_batch_step_timed(self._h, int(n), C.byref(ms))
        if rc != 0:
            raise MosesError(rc, self._L.moses_batch_last_error(self._h).decode())
        return ms.value

    @property
    def tiles(self) -> int:
        return self._L.moses_batch_tiles(self._h)

    def tile_rows(self):
        """(rows of the chosen 32-wide tile shape, [ms of one first stage for
        32 x 4, 32 x 8, 32 x 16]) as timed by moses_batch_create."""
        ms = np.zeros(3)
        ty = self._L.moses_batch_tile_rows(self._h, _p(ms))
        return ty, [float(x) for x in ms]

    def set_tile_rows(self, rows: int):
        rc = self._L.moses_batch_set_tile_rows(self._h, int(rows))
        if rc != 0:
            raise MosesError(rc, self._L.moses_batch_last_error(self._h).decode())

    def debug_timeout(self, on: bool = True):
        """Make every wait of the launch's grid barrier run out (testing the
        MOSES_ETIMEOUT path without a fault); False restores normal steps."""
        rc = self._L.moses_batch_debug_timeout(self._h, int(bool(on)))
        if rc != 0:
            raise MosesError(rc, self._L.moses_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._L.moses_batch_destroy(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def from_config(cfg: dict, precision: int = FP64, stream=None) -> Sim:
    """GPU simulation of a workload dict from ``workloads``."""
    s = Sim(cfg["dem"], cfg["dx"], cfg["dy"], cfg["params"], precision=precision, stream=stream)
    s.set_release(cfg["h"], cfg["phi_s"], cfg.get("vx_s"), cfg.get("vy_s"), cfg.get("vx_f"), cfg.get("vy_f"))
    if cfg.get("inflow"):
        f = cfg["inflow"]
        s.set_inflow(f["side"], f["i0"], f["i1"], f["t"], f["Q"], f["phi"])
    return s


def debug_math(x) -> dict:
    """The stage kernels' reciprocal and square roots of the values x, beside
    CUDA's own (moses_debug_math)."""
    x = _f64(x).ravel()
    out = np.empty((9, x.size))
    rc = lib().moses_debug_math(_p(x), int(x.size), _p(out))
    if rc != 0:
        raise MosesError(rc, lib().moses_last_error(None).decode())
    names = ("frcp", "cuda_rcp", "fsqrt", "cuda_sqrt", "frsqrt", "cuda_rsqrt", "frcp32", "fsqrt32", "frsqrt32")
    return dict(zip(names, out))


def fp64_rate(reps: int = 5) -> float:
    """Measured FP64 FMA rate of the current device [TFLOP/s] (moses_debug_fp64_rate)."""
    t = C.c_double()
    rc = lib().moses_debug_fp64_rate(int(reps), C.byref(t))
    if rc != 0:
        raise MosesError(rc, lib().moses_last_error(None).decode())
    return t.value


def flux_eval(n: int = 1 << 22, reps: int = 10) -> dict:
    """The central face flux in FP64 and in double-float arithmetic (pairs of
    FP32 numbers; not IEEE FP64) on n synthetic faces (moses_debug_flux_eval):
    face fluxes per second of each form and the double-float fluxes' relative
    max-norm and largest relative difference against the FP64 ones."""
    r = np.zeros(4)
    rc = lib().moses_debug_flux_eval(int(n), int(reps), _p(r))
    if rc != 0:
        raise MosesError(rc, lib().moses_last_error(None).decode())
    return {"f64_gfaces_per_s": float(r[0]), "df_gfaces_per_s": float(r[1]),
            "relmax_vs_f64": float(r[2]), "max_rel_vs_f64": float(r[3])}


def version() -> str:
    return lib().moses_version().decode()


def deposit_misfit(cfg: dict, h0, delta_b_deg, c_d, phi_int_deg, hs_target, nsteps: int, ckpt_every: int = 0,
                   precision: int = FP32):
    """Deposit misfit L = sum (h^s(t_N) - h^s_target)^2 dx dy as a differentiable
    torch function of the release thickness h0, the basal friction angle
    delta_b (degrees), the drag coefficient c_D and the internal friction
    angle phi_int (degrees; it enters the model through the Savage-Hutter
    earth-pressure coefficients when cfg's k_mode is 1, else its gradient is 0).

    The forward pass and the gradients both come from moses_adjoint_misfit
    (one forward run, checkpointed recomputation, reverse sweep); backward
    scales the stored gradients by the incoming gradient.
    """
    import torch

    class _Misfit(torch.autograd.Function):
        @staticmethod
        def forward(ctx, h0_t, db_t, cd_t, pi_t):
            params = dict(cfg["params"], delta_b_deg=float(db_t), c_d=float(cd_t), phi_int_deg=float(pi_t))
            sim = Sim(cfg["dem"], cfg["dx"], cfg["dy"], params, precision=precision)
            try:
                sim.set_release(h0_t.detach().cpu().double().numpy(), cfg["phi_s"])
                r = sim.adjoint_misfit(nsteps, hs_target, ckpt_every=ckpt_every, release_phi=cfg["phi_s"])
            finally:
                sim.close()
            gh = torch.from_numpy(r["g_release_h"]).to(h0_t.device, h0_t.dtype)
            gp = torch.tensor(r["g_params"], dtype=torch.float64)
            ctx.save_for_backward(gh, gp)
            return torch.tensor(r["loss"], dtype=torch.float64)

        @staticmethod
        def backward(ctx, gout):
            gh, gp = ctx.saved_tensors
            g = gout.to(torch.float64)
            return (gout.to(gh.dtype) * gh, (g * gp[0]).to(torch.float64), (g * gp[2]).to(torch.float64),
                    (g * gp[1]).to(torch.float64))

    return _Misfit.apply(h0, delta_b_deg, c_d, phi_int_deg)
