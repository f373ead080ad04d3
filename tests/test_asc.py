"""ESRI ASCII grid and hydrograph files (host side, no GPU)."""
import numpy as np
import pytest

from oracle.oracle import from_config as oracle_from_config
from paper_2104_06784_gb300 import asc, workloads as W


def test_round_trip_and_orientation(tmp_path):
    g = np.arange(12, dtype=float).reshape(3, 4) * 0.5  # row 0 = south
    p = tmp_path / "g.asc"
    asc.write_asc(str(p), g, 5.0, xll=100.0, yll=200.0)
    lines = p.read_text().splitlines()
    assert lines[0] == "ncols 4" and lines[1] == "nrows 3"
    # the first data row of the file is the northern one
    assert [float(v) for v in lines[6].split()] == list(g[2])
    back, hdr = asc.read_asc(str(p))
    assert np.array_equal(back, g)
    assert hdr["dx"] == hdr["dy"] == 5.0 and hdr["xll"] == 100.0 and hdr["yll"] == 200.0


def test_nodata_and_header_variants(tmp_path):
    p = tmp_path / "v.asc"
    p.write_text("NCOLS 3\nNROWS 2\nXLLCENTER 2.5\nYLLCENTER 2.5\nCELLSIZE 5\nNODATA_VALUE -9999\n"
                 "1 2 -9999\n4 5 6\n")
    g, hdr = asc.read_asc(str(p))
    assert hdr["xll"] == 0.0 and hdr["yll"] == 0.0
    assert g[0].tolist() == [4.0, 5.0, 6.0]
    assert g[1, 0] == 1.0 and np.isnan(g[1, 2])
    g0, _ = asc.read_asc(str(p), nodata=0.0)
    assert g0[1, 2] == 0.0
    # rectangular cells
    q = tmp_path / "r.asc"
    asc.write_asc(str(q), g0, 5.0, 10.0)
    _, h2 = asc.read_asc(str(q))
    assert (h2["dx"], h2["dy"]) == (5.0, 10.0)


@pytest.mark.parametrize("text", [
    "ncols 2\nnrows 2\ncellsize 1\n1 2 3\n",          # too few values
    "ncols 2\nnrows 2\n1 2 3 4\n",                    # no cell size
    "ncols 2.5\nnrows 2\ncellsize 1\n1 2 3 4 5\n",    # non-integer size
    "ncols 2\nnrows 2\ncellsize -1\n1 2 3 4\n",       # negative cell size
])
def test_malformed_grids_are_rejected(tmp_path, text):
    p = tmp_path / "bad.asc"
    p.write_text(text)
    with pytest.raises(ValueError):
        asc.read_asc(str(p))


def test_hydrograph(tmp_path):
    p = tmp_path / "q.txt"
    p.write_text("# t Q phi\n0 0 0.5\n60, 800, 0.5\n300 0 0.5\n")
    t, Q, phi = asc.read_hydrograph(str(p))
    assert t.tolist() == [0, 60, 300] and Q.tolist() == [0, 800, 0] and phi.tolist() == [0.5] * 3
    p.write_text("0 0\n10 5\n5 1\n")
    with pytest.raises(ValueError):
        asc.read_hydrograph(str(p))


def test_config_from_asc_runs_like_the_array_config(tmp_path):
    cfg = W.release_config(nx=24, ny=20)
    asc.write_asc(str(tmp_path / "dem.asc"), cfg["dem"], cfg["dx"], fmt="%.17g")
    asc.write_asc(str(tmp_path / "h.asc"), cfg["h"], cfg["dx"], fmt="%.17g")
    asc.write_asc(str(tmp_path / "phi.asc"), cfg["phi_s"], cfg["dx"], fmt="%.17g")
    c2 = asc.config_from_asc(str(tmp_path / "dem.asc"), cfg["params"], str(tmp_path / "h.asc"),
                             str(tmp_path / "phi.asc"))
    for k in ("dem", "h", "phi_s"):
        assert np.array_equal(c2[k], cfg[k])
    a, b = oracle_from_config(cfg), oracle_from_config(c2)
    a.step(3)
    b.step(3)
    assert np.array_equal(a.get_U(), b.get_U())
    # output fields as .asc
    st = dict(zip(("h", "phi_s", "vx_s", "vy_s", "vx_f", "vy_f"), [np.ones((20, 24)) * q for q in range(6)]))
    paths = asc.write_state_asc(st, str(tmp_path / "out"), cfg["dx"])
    assert len(paths) == 6 and np.array_equal(asc.read_asc(paths[3])[0], st["vy_s"])


def test_dem_with_nodata_is_rejected(tmp_path):
    g = np.zeros((3, 3))
    g[1, 1] = np.nan
    asc.write_asc(str(tmp_path / "d.asc"), g, 1.0)
    with pytest.raises(ValueError):
        asc.config_from_asc(str(tmp_path / "d.asc"), W.default_params())
