"""The premise of wet/dry masking, pinned on the oracle (no GPU).

A cell with no mass within the reach of the stencil has the zero state as its
result, exactly, whatever momenta its massless neighbours carry: its face
states are dry (velocities 0 by the dry rule), so its fluxes, pressures and
speeds are 0, and its sources scale with masses or velocities.  The stepping
kernels write that zero state instead of computing it.

The kernels take a tile as wet when its cells or a 2-cell halo hold mass, the
data reach of one stage: a face value uses the slopes of the two cells beside
it (Sect. 2.2).  With minmod the values reach only 1 cell per stage.  A dry
cell next to a dry cell has a zero slope, since minmod(0, x) = 0, so the face
between two dry cells has zero states on both sides.  A two-step modified
Euler step therefore reaches 2 cells and a three-stage Runge-Kutta step 3;
these tighter reaches are pinned here for both fluxes.  The WENO3 face values
are pinned at the kernels' 2-cell reach per stage.

The oracle computes every cell of the grid in plain loops, so this is a
property of the scheme, not of the kernels.  The cases run with and without
momenta on massless cells.
"""
import numpy as np
import pytest

from oracle.oracle import from_config
from paper_2104_06784_gb300 import workloads as W


def _dilate(m, r):
    """Cells within Chebyshev distance r of a True cell (clipped at the edge)."""
    d = m.copy()
    for s in range(1, r + 1):
        d[:, s:] |= m[:, :-s]
        d[:, :-s] |= m[:, s:]
    e = d.copy()
    for s in range(1, r + 1):
        e[s:, :] |= d[:-s, :]
        e[:-s, :] |= d[s:, :]
    return e


def _case(nx, ny, seed, bc, momenta_on_dry, **over):
    rng = np.random.default_rng(seed)
    dem = W.spectral_dem(nx, ny, 5.0, 2.2, 40.0, seed=seed) + rng.random((ny, nx))
    U = np.zeros((6, ny, nx))
    for _ in range(6):  # isolated wet cells and small wet patches, some on the edges
        j, i = int(rng.integers(0, ny)), int(rng.integers(0, nx))
        if rng.random() < 0.3:
            j = 0 if rng.random() < 0.5 else ny - 1
        hj, hi = int(rng.integers(1, 4)), int(rng.integers(1, 4))
        h = rng.uniform(0.2, 1.5, (min(hj, ny - j), min(hi, nx - i)))
        sl = (slice(j, j + hj), slice(i, i + hi))
        U[0][sl], U[3][sl] = 0.6 * h, 0.4 * h
        for c in (1, 2, 4, 5):
            U[c][sl] = U[3 * (c // 3)][sl] * rng.normal(0.0, 2.0, h.shape)
    mass = (U[0] != 0) | (U[3] != 0)
    if momenta_on_dry:  # not a physical state; the dry rule zeroes these momenta
        for c in (1, 2, 4, 5):
            U[c] = np.where(~mass & (rng.random((ny, nx)) < 0.3), rng.normal(0.0, 1.0, (ny, nx)), U[c])
    cfg = dict(name="masking", dem=dem, dx=5.0, dy=5.0, params=W.default_params(bc=bc, **over),
               h=np.zeros((ny, nx)), phi_s=np.zeros((ny, nx)))
    return cfg, U, mass


def _zero_beyond(out, mass, r):
    far = ~_dilate(mass, r)
    assert far.any() and (~far).any()
    assert np.all(out[:, far] == 0.0), r
    assert np.any(out[:, ~far] != 0.0)


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 1, 1), (0, 1, 1, 0)])
@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("momenta_on_dry", [False, True])
def test_stage_and_step_are_zero_beyond_the_reach(bc, scheme, momenta_on_dry):
    nx, ny = 61, 47
    cfg, U, mass = _case(nx, ny, 17 + 3 * scheme + bc[1], bc, momenta_on_dry, scheme=scheme)
    o = from_config(cfg)
    o.set_U(U)
    _zero_beyond(o.stage(0.0, 0.02), mass, 1)
    o.set_U(U)
    o.step_dt(0.02)
    _zero_beyond(o.get_U(), mass, 2)


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 1, 1)])
def test_three_stage_step_is_zero_beyond_the_reach(bc):
    nx, ny = 61, 47
    cfg, U, mass = _case(nx, ny, 29 + bc[0], bc, False, rk=3)
    o = from_config(cfg)
    o.set_U(U)
    o.step_dt(0.02)
    _zero_beyond(o.get_U(), mass, 3)


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (0, 1, 1, 0)])
@pytest.mark.parametrize("momenta_on_dry", [False, True])
def test_weno_stage_and_step_are_zero_beyond_the_halo(bc, momenta_on_dry):
    nx, ny = 61, 47
    cfg, U, mass = _case(nx, ny, 41 + bc[1], bc, momenta_on_dry, recon=1)
    o = from_config(cfg)
    o.set_U(U)
    _zero_beyond(o.stage(0.0, 0.02), mass, 2)
    o.set_U(U)
    o.step_dt(0.02)
    _zero_beyond(o.get_U(), mass, 4)
