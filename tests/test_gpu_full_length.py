"""The two long workloads at their full length, scaled down in cells so that
the oracle finishes in seconds: the large-release event (spectral DEM, the
event's recipe at 96 x 80 cells of 10 m) for its 10 000 steps, and the
channel-and-fan inflow (64 x 32 cells of 20 m, the same 100 m inlet and
hydrograph) to t = 600 s, both forms against the FP64 oracle.

Over thousands of steps the flows reach states in which a rounding
difference grows: cells stop or start on a knife edge, and at the end of
the inflow run the fluid phase has drained to thin films (its largest mass
is 0.4 % of the solid's).  For each field the test therefore measures how
far the oracle itself moves from its own run when its state is disturbed
after every step -- by one ulp for the FP64 form, by the rounding to FP32
for the FP32 form -- and holds the GPU run to the form's tolerance
(1e-10 relative max-norm per conserved component for FP64; 2e-4 relative
L1 on depth and velocities, velocities on cells deeper than 1 cm, for
FP32), or to 10 times that sensitivity where it exceeds a tenth of the
tolerance.  The mass drift of both forms stays within 1e-7 in every case.
"""
import numpy as np
import pytest

from oracle.oracle import from_config as oracle_from_config
from paper_2104_06784_gb300 import moses, workloads as W
from tests.test_gpu_parity import _fields, rel_l1

pytestmark = pytest.mark.gpu

T_END = 600.0
FIELDS = ("h", "vx_s", "vy_s", "vx_f", "vy_f")


def _inflow():
    return W.inflow_config(nx=64, ny=32, dx=20.0, inlet_cells=5)


def _release():
    return W.large_release_config(n=96, ny=80, dx=10.0, seed=2, volume=2e5, radius_cells=8)


def _oracle_until(o, t_end, disturb=None):
    """Oracle steps (CFL time steps, the last one shortened to land on
    t_end); `disturb(U)` is applied to the state after every step."""
    while o.t < t_end:
        dt = o.cfl_dt()
        if o.t + dt >= t_end:
            o.step_dt(t_end - o.t)
        else:
            o.step(1)
        if disturb is not None:
            o.set_U(disturb(o.get_U()))


def _oracle_steps(o, n, disturb=None):
    for _ in range(n):
        o.step(1)
        if disturb is not None:
            o.set_U(disturb(o.get_U()))


def _field_errors(U, Uo, J, hd, h_min=0.01):
    hg, vg, pg = _fields(U, J, hd)
    ho, vo, po = _fields(Uo, J, hd)
    e = {"h": rel_l1(hg, ho)}
    for name, a, b, da, db in zip(FIELDS[1:], vg, vo, pg, po):
        deep = (da > h_min) & (db > h_min)
        e[name] = rel_l1(a[deep], b[deep])
    return e


def _componentwise(U, Uo):
    scale = np.abs(Uo).reshape(6, -1).max(axis=1)
    scale = np.where(scale > 0, scale, 1.0)
    return np.abs(U - Uo).reshape(6, -1).max(axis=1) / scale


_ORACLE = {}  # case -> the oracle's own final state (shared by the two forms' tests)


def _runs(cfg, inflow, precision):
    """The GPU run, the oracle's own final state, and the final states of the
    oracle's two disturbed runs."""
    advance = (lambda s, d=None: _oracle_until(s, T_END, d)) if inflow else (lambda s, d=None: _oracle_steps(s, 10000, d))
    case = "inflow" if inflow else "release"
    if case not in _ORACLE:
        o = oracle_from_config(cfg)
        advance(o)
        _ORACLE[case] = (o.get_U(), o.geometry()["J"])
    if precision == moses.FP64:
        rngs = [np.random.default_rng(k) for k in (1, 2)]
        disturbs = [lambda U, r=r: U * (1.0 + 2.0 ** -52 * r.uniform(-1.0, 1.0, U.shape)) for r in rngs]
    else:
        rng = np.random.default_rng(3)
        disturbs = [lambda U: U.astype(np.float32).astype(np.float64),
                    lambda U: (U * (1.0 + 2.0 ** -24 * rng.uniform(-1.0, 1.0, U.shape))).astype(np.float32).astype(np.float64)]
    others = []
    for d in disturbs:
        r = oracle_from_config(cfg)
        advance(r, d)
        others.append(r.get_U())
    g = moses.from_config(cfg, precision=precision)
    b0 = g.budget()
    if inflow:
        g.run_until(T_END)
    else:
        g.step(10000)
    return g, _ORACLE[case], others, b0


def _drift(g, b0):
    b = g.budget()
    return max(abs(b[f"vol_{p}"] - b0[f"vol_{p}"] - b[f"bnd_in_{p}"] - b[f"clamp_{p}"]) / b[f"vol_{p}"]
               for p in ("s", "f"))


@pytest.mark.parametrize("case", ["release", "inflow"])
def test_full_length_fp64(case):
    inflow = case == "inflow"
    cfg = _inflow() if inflow else _release()
    g, (Uo, J), others, b0 = _runs(cfg, inflow, moses.FP64)
    sens = np.max([_componentwise(U, Uo) for U in others], axis=0)
    err = _componentwise(g.get_conserved(), Uo)
    for c in range(6):
        lim = 1e-10 if sens[c] <= 1e-11 else max(1e-10, 10.0 * sens[c])
        assert err[c] <= lim, f"FP64 {case}: component {c} {err[c]:.3e} (oracle's own sensitivity {sens[c]:.3e})"
    # the depth field in L1, whatever the conditioning of the thin films
    hd = cfg["params"]["h_dry"]
    assert _field_errors(g.get_conserved(), Uo, J, hd)["h"] <= 1e-9
    assert _drift(g, b0) <= 1e-7


@pytest.mark.parametrize("case", ["release", "inflow"])
def test_full_length_fp32(case):
    inflow = case == "inflow"
    cfg = _inflow() if inflow else _release()
    g, (Uo, J), others, b0 = _runs(cfg, inflow, moses.FP32)
    hd = cfg["params"]["h_dry"]
    err = _field_errors(g.get_conserved(), Uo, J, hd)
    sens = {k: max(_field_errors(U, Uo, J, hd)[k] for U in others) for k in FIELDS}
    for k in FIELDS:
        lim = 2e-4 if sens[k] <= 2e-5 else max(2e-4, 10.0 * sens[k])
        assert err[k] <= lim, f"FP32 {case}: {k} {err[k]:.3e} (oracle's own sensitivity {sens[k]:.3e})"
    assert _drift(g, b0) <= 1e-7
