"""The earth-pressure form (k_mode 1, reading R10) on the GPU against the FP64
oracle, element by element.

The Savage-Hutter coefficient multiplies the solid pressure of each direction
and the solid celerity; a cell takes K_pass where it and its two neighbours
along the axis carry solid and the solid velocity falls along the axis,
K_act otherwise.  The kernels decide with the same IEEE operations as the
oracle (correctly rounded division and subtraction), so from the same input
they take the same branch at every face, and a dead band (a velocity drop
of more than 1e-6 of the two speeds plus 1e-6 m/s counts as compression)
keeps rounding noise at cells between neighbours at rest from flipping it.
Tolerances as in test_gpu_parity.py: 1e-10 relative max-norm (FP64), 2e-4
relative L1 on depth and velocities (FP32); where the switch makes a run
sensitive to rounding (a pile coming to rest, FP32 state), the bar is ten
times the oracle's own measured sensitivity to that rounding when that is
larger.
"""
import numpy as np
import pytest

from oracle.oracle import from_config as oracle_from_config
from paper_2104_06784_gb300 import moses, workloads as W
from tests.test_gpu_parity import TOL64, _fp32_sensitivity, _fp32_vs_oracle, both, fp64_sensitivity, rel_maxnorm

pytestmark = pytest.mark.gpu


def _random_case(nx, ny, bc, seed, **over):
    rng = np.random.default_rng(seed)
    dem = W.spectral_dem(nx, ny, 5.0, 2.2, 40.0, seed=seed) + rng.random((ny, nx))
    p = W.default_params(bc=bc, k_mode=1, **over)
    return dict(name="random", dem=dem, dx=5.0, dy=5.0, params=p, **W.random_state(nx, ny, seed=seed + 1))


@pytest.mark.parametrize("nx,ny", [(77, 53), (33, 9), (5, 70), (1, 17), (23, 1)])
@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 1, 1), (0, 1, 1, 0)])
def test_stage_parity_fp64(nx, ny, bc):
    cfg = _random_case(nx, ny, bc, seed=nx * 101 + ny)
    g, o = both(cfg)
    for t, dt in ((0.0, 0.01), (3.0, 0.05)):
        err = rel_maxnorm(g.stage(t, dt), o.stage(t, dt))
        assert err < TOL64, f"earth-pressure stage parity {err} ({nx}x{ny}, bc={bc})"
    assert abs(g.max_speed() - o.max_speed()) <= 1e-13 * o.max_speed()
    if nx > 2 and ny > 2:  # the coefficient acts on these states
        o0 = oracle_from_config(dict(cfg, params=dict(cfg["params"], k_mode=0)))
        assert rel_maxnorm(o0.stage(0.0, 0.01), o.stage(0.0, 0.01)) > 1e-6


@pytest.mark.parametrize("tile", [0, 1, 2, 3])
def test_stage_parity_every_tile(tile):
    cfg = _random_case(70, 37, (0, 1, 1, 0), seed=5)
    g, o = both(cfg)
    g.set_tile(tile)
    assert rel_maxnorm(g.stage(1.0, 0.02), o.stage(1.0, 0.02)) < TOL64


@pytest.mark.parametrize("tile", [0, 1, 2, 3])
def test_masked_steps_fp64(tile):
    """moses_step (wet/dry classification and the listed tiles) with the
    earth-pressure form: a pile in a mostly dry domain, 60 steps."""
    cfg = W.release_config(nx=77, ny=61, cfl=0.3, k_mode=1)
    g, o = both(cfg)
    g.set_tile(tile)
    g.step(60)
    o.step(60)
    assert rel_maxnorm(g.get_conserved(), o.get_U()) < TOL64


def test_release_trajectory_fp64_cfl05():
    """The arc-plane release (128 x 128, closed, CFL 0.5, 2000 steps) with
    internal friction: phi_int = 35 deg, delta_b = 25 deg (K_act 0.705,
    K_pass 3.256).  The regime switch is a jump in the flux; while the pile
    comes to rest at CFL 0.5 (above the scheme's positivity limit) cells sit
    at the switch and at the stopping condition, and the FP64 oracle alone,
    perturbed by one ulp per step, leaves its own run by a few 1e-8 at step
    2000 (measured; 1e-11 through step 1500).  Each mark is held to
    max(1e-10, 10 x that sensitivity): 1e-10 until the pile stops."""
    cfg = W.release_config(k_mode=1)
    g, o = both(cfg)
    marks = (10, 100, 500, 1000, 1500, 2000)
    sens = fp64_sensitivity(cfg, marks)
    done = 0
    for m in marks:
        g.step(m - done)
        o.step(m - done)
        done = m
        err = rel_maxnorm(g.get_conserved(), o.get_U())
        lim = max(TOL64, 10.0 * sens[m])
        assert err < lim, f"earth-pressure trajectory departs at step {m}: {err} (sensitivity {sens[m]})"
        # the time steps follow the state: the clock as closely as the state
        assert abs(g.budget()["t"] - o.t) <= max(1e-12, 10.0 * sens[m]) * o.t
    # internal friction changes the run
    o0 = oracle_from_config(W.release_config(k_mode=0))
    o0.step(100)
    o1 = oracle_from_config(cfg)
    o1.step(100)
    assert rel_maxnorm(o1.get_U(), o0.get_U()) > 1e-3


def test_rk3_trajectory_fp64():
    cfg = W.release_config(nx=64, ny=64, cfl=0.2, k_mode=1, rk=3)
    g, o = both(cfg)
    g.step(200)
    o.step(200)
    assert rel_maxnorm(g.get_conserved(), o.get_U()) < TOL64


def test_spectral_release_fp64():
    cfg = W.large_release_config(n=150, ny=131, dx=10.0, seed=3, volume=2e5, radius_cells=8, k_mode=1)
    g, o = both(cfg)
    g.step(150)
    o.step(150)
    assert rel_maxnorm(g.get_conserved(), o.get_U()) < TOL64


@pytest.mark.parametrize("case", ["spectral", "arc"])
def test_trajectory_fp32(case):
    """FP32 state and fluxes (FP64 budgets and stopping test) with the
    earth-pressure form: depth and velocities (cells deeper than 1 cm) within
    max(2e-4, 10 x the oracle's own FP32 sensitivity) relative L1 of the FP64
    oracle (the regime switch lets FP32 rounding move a cell across it; the
    sensitivity is how far the oracle moves with its state rounded to FP32
    after each step), mass drift within 1e-7."""
    if case == "spectral":
        cfg, marks = W.large_release_config(n=192, ny=160, dx=10.0, seed=2, volume=1e6, radius_cells=12,
                                            k_mode=1), (150, 400)
    else:
        cfg, marks = W.release_config(cfl=0.1, k_mode=1), (300, 800)
    sens = _fp32_sensitivity(cfg, marks)
    for m, errs in _fp32_vs_oracle(cfg, marks).items():
        for k, v in errs.items():
            lim = 1e-7 if k == "drift" else max(2e-4, 10.0 * sens[m][k])
            assert v <= lim, f"FP32 {k} {v} at step {m} ({case}; sensitivity {sens[m].get(k)})"


def test_forms_without_earth_pressure_are_rejected():
    base = W.release_config(nx=20, ny=20, k_mode=1)
    for over in (dict(scheme=1), dict(recon=1), dict(nu_f=1.0), dict(phi_int_deg=20.0, delta_b_deg=25.0)):
        with pytest.raises(moses.MosesError):
            moses.from_config(dict(base, params=dict(base["params"], **over)))
    a = moses.from_config(base)
    with pytest.raises(moses.MosesError):
        moses.Batch([a])
