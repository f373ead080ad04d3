"""Host-side logic of bench.py (no GPU): the wet-tile fraction that the line
reports per window, the roofline's bytes per computed cell-step, and the
clock sampler's window summary."""
import time

import numpy as np

import bench


def _brute_wet_tiles(U, tx, ty):
    """A tile computes if a cell of it or within 2 cells of it has mass."""
    ny, nx = U.shape[1:]
    m = (U[0] != 0) | (U[3] != 0)
    wet = []
    for by in range(0, ny, ty):
        for bx in range(0, nx, tx):
            y0, y1 = max(by - 2, 0), min(by + ty + 2, ny)
            x0, x1 = max(bx - 2, 0), min(bx + tx + 2, nx)
            wet.append(m[y0:y1, x0:x1].any())
    return float(np.mean(wet))


def test_wet_tile_fraction_matches_brute_force():
    rng = np.random.default_rng(3)
    for nx, ny, tx, ty in ((97, 41, 32, 8), (64, 64, 32, 4), (130, 35, 32, 16), (5, 3, 32, 8)):
        U = np.zeros((6, ny, nx))
        for _ in range(4):
            j, i = rng.integers(0, ny), rng.integers(0, nx)
            U[3 * rng.integers(0, 2), j, i] = 1.0
        assert bench.wet_tile_fraction(U, tx, ty) == _brute_wet_tiles(U, tx, ty)
    # a mass two cells from a tile edge reaches the neighbour, three cells does not
    U = np.zeros((6, 16, 64))
    U[0, 5, 33] = 1.0  # tile column 1 (x 32..63): 1 from the edge
    assert bench.wet_tile_fraction(U, 32, 8) == 0.5
    U[0, 5, 33] = 0.0
    U[0, 5, 35] = 1.0  # 3 from the edge: its own column only
    assert bench.wet_tile_fraction(U, 32, 8) == 0.25


def test_clock_summary_window_and_bracketing():
    s = bench.ClockSampler(0)
    t = time.time()
    row = "0, {mhz}, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, {cap}"
    s.lines = [(t - 0.05, row.format(mhz=2070, cap="Not Active")),
               (t + 0.01, row.format(mhz=1980, cap="Active")),
               (t + 0.50, row.format(mhz=2070, cap="Not Active"))]
    s.windows = [[t, t + 0.02]]
    got = s.summary()
    assert got["samples"] == 1 and got["sm_mhz"] == 1980 and got["reasons"] == ["sw_power_cap"]
    assert got["window"] == "in the timed window"
    # a window shorter than the interval that caught no sample: the two around it
    s.lines = [s.lines[0], s.lines[2]]
    got = s.summary()
    assert got["samples"] == 2 and "bracketing" in got["window"]
    s.lines = []
    assert s.summary()["reasons"] == ["unsampled"]


def test_roofline_bytes_per_computed_cell_step():
    """The roofline's HBM bytes: 13 words per computed cell-step (read U^n, write
    U^{n+1}, read the bed), FP64 104 B and FP32 52 B."""
    assert bench.cell_step_gbs(1e9, 8, 1.0) == 104.0
    assert bench.cell_step_gbs(1e9, 4, 0.5) == 104.0
    assert bench._traffic("f64", "no-such-source", 10) is None
