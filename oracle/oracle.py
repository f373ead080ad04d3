"""ctypes wrapper of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use this module; the library itself never
does.  It shares nothing with the CUDA library; the two meet only through the
seeded inputs of ``paper_2104_06784_gb300.workloads``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lib = None


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile oracle.c with plain -O2, no FMA contraction, no fast-math.

    openmp=True builds the copy that runs the loops over rows on every host
    core (-fopenmp), for timing the multi-core CPU baseline only; the tests
    use the plain build."""
    out = _LIB_OMP if openmp else _LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               *(["-fopenmp"] if openmp else []), "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def lib_openmp():
    """The -fopenmp build of the oracle (multi-core CPU baseline timing)."""
    return load(build(openmp=True))


class _Params(C.Structure):
    _fields_ = [("g", C.c_double), ("eps", C.c_double), ("eps_chi", C.c_double),
                ("rho_s", C.c_double), ("rho_f", C.c_double),
                ("delta_b_deg", C.c_double), ("phi_int_deg", C.c_double), ("k_mode", C.c_int),
                ("c_d", C.c_double), ("nu_f", C.c_double), ("k_f", C.c_double),
                ("cfl", C.c_double), ("dt_max", C.c_double), ("h_dry", C.c_double),
                ("bc", C.c_int * 4), ("fluid_pg_mode", C.c_int), ("scheme", C.c_int), ("recon", C.c_int),
                ("rk", C.c_int)]


def _params(p: dict) -> _Params:
    s = _Params()
    for name, _ in _Params._fields_:
        if name == "bc":
            s.bc[:] = [int(v) for v in p["bc"]]
        elif name in ("k_mode", "fluid_pg_mode"):
            setattr(s, name, int(p[name]))
        elif name in ("scheme", "recon", "rk"):
            setattr(s, name, int(p.get(name, 2 if name == "rk" else 0)))
        else:
            setattr(s, name, float(p[name]))
    return s


def load(path: str):
    """Load an oracle library from `path` (the default build, or a copy with a
    planted mistake compiled by the mutation tests)."""
    L = C.CDLL(path)
    _declare(L)
    return L


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = load(_LIB)
    return _lib


def _declare(L):
    """ctypes signatures of the oracle's entry points."""
    dp = C.POINTER(C.c_double)
    vp = C.c_void_p
    L.orc_create.argtypes = [dp, C.c_int, C.c_int, C.c_double, C.c_double, C.POINTER(_Params),
                             C.POINTER(vp)]
    L.orc_destroy.argtypes = [vp]
    L.orc_set_U.argtypes = [vp, dp]
    L.orc_get_U.argtypes = [vp, dp]
    L.orc_set_release.argtypes = [vp, dp, dp, dp, dp, dp, dp]
    L.orc_set_inflow.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, dp, dp, dp]
    L.orc_set_time.argtypes = [vp, C.c_double]
    L.orc_get_time.argtypes = [vp]
    L.orc_get_time.restype = C.c_double
    L.orc_last_dt.argtypes = [vp]
    L.orc_last_dt.restype = C.c_double
    L.orc_max_speed.argtypes = [vp]
    L.orc_max_speed.restype = C.c_double
    L.orc_max_speed_rows.argtypes = [vp, C.c_int, C.c_int]
    L.orc_max_speed_rows.restype = C.c_double
    L.orc_cfl_dt.argtypes = [vp]
    L.orc_cfl_dt.restype = C.c_double
    L.orc_step.argtypes = [vp, C.c_int, dp]
    L.orc_step_dt.argtypes = [vp, C.c_double]
    L.orc_step_amax.argtypes = [vp, C.c_double]
    L.orc_step_amax.restype = C.c_double
    L.orc_stage.argtypes = [vp, C.c_double, C.c_double, dp]
    L.orc_budget.argtypes = [vp, dp]
    L.orc_geometry.argtypes = [vp, dp]
    L.orc_kappa.argtypes = [vp, C.c_int, C.c_int, C.c_double, C.c_double]
    L.orc_kappa.restype = C.c_double
    L.orc_tangential.argtypes = [vp, C.c_int, C.c_int, C.c_double, C.c_double, dp]
    L.orc_inflow_state.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_double, dp]
    L.orc_cell_geom.argtypes = [vp, C.c_int, C.c_int, dp]
    L.orc_earth_pressure.argtypes = [C.POINTER(_Params), dp]


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


BUDGET_KEYS = ("vol_s", "vol_f", "mom_xs", "mom_ys", "mom_xf", "mom_yf", "bnd_in_s", "bnd_in_f",
               "clamp_s", "clamp_f", "clamp_cells", "t", "steps")


class OracleSim:
    """One simulation held by the oracle.  Arrays are ``[j, i]`` (south row
    first); the conserved state U is ``(6, ny, nx)`` with U1 = J h^s,
    U2 = J h^s v_X^s, U3 = J h^s v_Y^s, U4 = J h^f, U5 = J h^f v_X^f,
    U6 = J h^f v_Y^f."""

    def __init__(self, dem, dx: float, dy: float, params: dict, library=None):
        self._L = L = library if library is not None else lib()
        self.dem = _f64(dem)
        self.ny, self.nx = self.dem.shape
        self.dx, self.dy = float(dx), float(dy)
        self.params = dict(params)
        self._p = _params(params)
        h = C.c_void_p()
        rc = L.orc_create(_ptr(self.dem), self.nx, self.ny, self.dx, self.dy, C.byref(self._p), C.byref(h))
        if rc != 0:
            raise ValueError(f"orc_create failed ({rc})")
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None):
            self._L.orc_destroy(self._h)
            self._h = None

    # state ------------------------------------------------------------------
    def set_U(self, U):
        U = _f64(U)
        assert U.shape == (6, self.ny, self.nx)
        self._L.orc_set_U(self._h, _ptr(U))

    def get_U(self) -> np.ndarray:
        U = np.empty((6, self.ny, self.nx))
        self._L.orc_get_U(self._h, _ptr(U))
        return U

    def set_release(self, h, phi_s, vx_s=None, vy_s=None, vx_f=None, vy_f=None):
        arrs = [_f64(a) if a is not None else None for a in (h, phi_s, vx_s, vy_s, vx_f, vy_f)]
        self._keep = arrs
        rc = self._L.orc_set_release(self._h, *[_ptr(a) for a in arrs])
        if rc != 0:
            raise ValueError("orc_set_release failed")

    def set_inflow(self, side: int, i0: int, i1: int, t, Q, phi):
        t, Q, phi = _f64(t), _f64(Q), _f64(phi)
        rc = self._L.orc_set_inflow(self._h, side, i0, i1, len(t), _ptr(t), _ptr(Q), _ptr(phi))
        if rc != 0:
            raise ValueError("orc_set_inflow failed")

    @property
    def t(self) -> float:
        return self._L.orc_get_time(self._h)

    @t.setter
    def t(self, v: float):
        self._L.orc_set_time(self._h, float(v))

    @property
    def last_dt(self) -> float:
        return self._L.orc_last_dt(self._h)

    # stepping ---------------------------------------------------------------
    def max_speed(self) -> float:
        return self._L.orc_max_speed(self._h)

    def max_speed_rows(self, j0: int, j1: int) -> float:
        """The largest cell speed over rows [j0, j1)."""
        return self._L.orc_max_speed_rows(self._h, int(j0), int(j1))

    def cfl_dt(self) -> float:
        return self._L.orc_cfl_dt(self._h)

    def step(self, n: int = 1) -> np.ndarray:
        dts = np.empty(max(n, 1))
        self._L.orc_step(self._h, n, _ptr(dts))
        return dts[:n]

    def step_dt(self, dt: float):
        self._L.orc_step_dt(self._h, float(dt))

    def step_amax(self, amax: float) -> float:
        """One step with the CFL time step of the given largest wave speed
        (a strip of a decomposed domain); returns the time step."""
        return self._L.orc_step_amax(self._h, float(amax))

    def stage(self, t: float, dt: float) -> np.ndarray:
        out = np.empty((6, self.ny, self.nx))
        self._L.orc_stage(self._h, float(t), float(dt), _ptr(out))
        return out

    # diagnostics ------------------------------------------------------------
    def budget(self) -> dict:
        out = np.empty(13)
        self._L.orc_budget(self._h, _ptr(out))
        return dict(zip(BUDGET_KEYS, out.tolist()))

    def geometry(self) -> dict:
        out = np.empty((15, self.ny, self.nx))
        self._L.orc_geometry(self._h, _ptr(out))
        names = ("J", "c", "nX", "nY", "nZ", "A11", "A12", "A21", "A22",
                 "dnX_dxi", "dnY_dxi", "dnZ_dxi", "dnX_deta", "dnY_deta", "dnZ_deta")
        return dict(zip(names, out))

    def kappa(self, i: int, j: int, vX: float, vY: float) -> float:
        return self._L.orc_kappa(self._h, i, j, float(vX), float(vY))

    def tangential(self, i: int, j: int, vX: float, vY: float):
        out = np.empty(2)
        self._L.orc_tangential(self._h, i, j, float(vX), float(vY), _ptr(out))
        return float(out[0]), float(out[1])

    def inflow_state(self, f: int, gi: int, gj: int, t: float) -> np.ndarray:
        out = np.empty(6)
        if self._L.orc_inflow_state(self._h, f, gi, gj, float(t), _ptr(out)) != 0:
            raise ValueError("no such inflow segment")
        return out

    def cell_geom(self, gi: int, gj: int) -> dict:
        out = np.empty(4)
        if self._L.orc_cell_geom(self._h, gi, gj, _ptr(out)) != 0:
            raise ValueError("cell out of range")
        return dict(zip(("J", "c", "A11", "A22"), out.tolist()))

    def primitive(self) -> dict:
        """h (normal thickness), phi_s and phase velocities from U, using the
        oracle's geometry (J) and the dry threshold."""
        U = self.get_U()
        J = self.geometry()["J"]
        hd = self.params["h_dry"]
        h = (U[0] + U[3]) / J
        wet = h > hd
        ws, wf = U[0] > J * hd, U[3] > J * hd
        with np.errstate(divide="ignore", invalid="ignore"):
            phi = np.where(wet, U[0] / (U[0] + U[3]), 0.0)
            out = dict(h=h, phi_s=phi,
                       vx_s=np.where(ws, U[1] / U[0], 0.0), vy_s=np.where(ws, U[2] / U[0], 0.0),
                       vx_f=np.where(wf, U[4] / U[3], 0.0), vy_f=np.where(wf, U[5] / U[3], 0.0))
        return out


def from_config(cfg: dict, library=None) -> OracleSim:
    """Oracle simulation of a workload dict from ``workloads``."""
    s = OracleSim(cfg["dem"], cfg["dx"], cfg["dy"], cfg["params"], library=library)
    s.set_release(cfg["h"], cfg["phi_s"], cfg.get("vx_s"), cfg.get("vy_s"), cfg.get("vx_f"), cfg.get("vy_f"))
    if cfg.get("inflow"):
        f = cfg["inflow"]
        s.set_inflow(f["side"], f["i0"], f["i1"], f["t"], f["Q"], f["phi"])
    return s


def earth_pressure(params: dict, library=None):
    """(K_act, K_pass) of a parameter set (reading R10; both 1 for k_mode 0)."""
    L = library if library is not None else lib()
    p = _params(params)
    out = np.empty(2)
    L.orc_earth_pressure(C.byref(p), _ptr(out))
    return float(out[0]), float(out[1])
