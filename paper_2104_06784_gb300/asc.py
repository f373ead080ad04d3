"""ESRI ASCII grids (.asc) for DEMs, release fields and results.

The paper's tool reads the DEM and the Mode-I initial configuration as
ESRI ASCII grids and writes its output fields in the same format for GIS
(Sect. 3.1.2 Stages 0 and 3).  A grid file is a header of keyword / value
lines -- ncols, nrows, xllcorner or xllcenter, yllcorner or yllcenter,
cellsize (or dx and dy), optionally NODATA_value -- followed by nrows rows of
ncols values, the northernmost row first.  The arrays of this package are
row-major with j = 0 the southern row (Y increasing north), so rows are
flipped on reading and on writing.

A Mode-II hydrograph file is a plain table with one sample per line: time
[s], discharge [m^3/s] and, optionally, the solid volume fraction; lines
starting with '#' are comments.

Host-side file handling only: no simulation arithmetic happens here.
"""
from __future__ import annotations

import os

import numpy as np

_KEYS = ("ncols", "nrows", "xllcorner", "yllcorner", "xllcenter", "yllcenter", "cellsize", "dx", "dy",
         "nodata_value")


def read_asc(path: str, nodata=np.nan):
    """Read an ESRI ASCII grid.  Returns (grid, header): grid of shape
    (nrows, ncols), float64, southern row first, NODATA cells set to
    `nodata`; header with ncols, nrows, dx, dy, xll, yll (the lower-left
    corner of the lower-left cell) and nodata_value (or None)."""
    hdr = {}
    with open(path) as f:
        lines = f.read().split("\n")
    k = 0
    while k < len(lines):
        parts = lines[k].split()
        if not parts:
            k += 1
            continue
        key = parts[0].lower()
        if key not in _KEYS:
            break
        if len(parts) != 2:
            raise ValueError(f"{path}: bad header line {lines[k]!r}")
        hdr[key] = float(parts[1])
        k += 1
    for need in ("ncols", "nrows"):
        if need not in hdr:
            raise ValueError(f"{path}: header lacks {need}")
    nx, ny = int(hdr["ncols"]), int(hdr["nrows"])
    if nx < 1 or ny < 1 or nx != hdr["ncols"] or ny != hdr["nrows"]:
        raise ValueError(f"{path}: ncols / nrows must be positive integers")
    if "cellsize" in hdr:
        dx = dy = hdr["cellsize"]
    elif "dx" in hdr and "dy" in hdr:
        dx, dy = hdr["dx"], hdr["dy"]
    else:
        raise ValueError(f"{path}: header lacks cellsize (or dx and dy)")
    if not (dx > 0 and dy > 0):
        raise ValueError(f"{path}: cell sizes must be > 0")
    if "xllcorner" in hdr:
        xll = hdr["xllcorner"]
    else:
        xll = hdr.get("xllcenter", 0.5 * dx) - 0.5 * dx
    if "yllcorner" in hdr:
        yll = hdr["yllcorner"]
    else:
        yll = hdr.get("yllcenter", 0.5 * dy) - 0.5 * dy
    vals = np.array(" ".join(lines[k:]).split(), dtype=np.float64)
    if vals.size != nx * ny:
        raise ValueError(f"{path}: expected {nx * ny} values, found {vals.size}")
    grid = vals.reshape(ny, nx)[::-1].copy()  # north-first rows -> south-first
    nd = hdr.get("nodata_value")
    if nd is not None:
        grid[grid == nd] = nodata
    return grid, dict(ncols=nx, nrows=ny, dx=dx, dy=dy, xll=xll, yll=yll, nodata_value=nd)


def write_asc(path: str, grid, dx: float, dy: float | None = None, xll: float = 0.0, yll: float = 0.0,
              nodata_value: float = -9999.0, fmt: str = "%.10g"):
    """Write a south-first (ny, nx) array as an ESRI ASCII grid (north row
    first).  Non-finite values are written as nodata_value.  With dx != dy
    the header uses dx / dy lines instead of cellsize."""
    a = np.asarray(grid, dtype=np.float64)
    if a.ndim != 2:
        raise ValueError("grid must be 2-D")
    dy = dx if dy is None else dy
    ny, nx = a.shape
    out = np.where(np.isfinite(a), a, nodata_value)[::-1]
    with open(path, "w") as f:
        f.write(f"ncols {nx}\nnrows {ny}\nxllcorner {xll!r}\nyllcorner {yll!r}\n")
        if dx == dy:
            f.write(f"cellsize {dx!r}\n")
        else:
            f.write(f"dx {dx!r}\ndy {dy!r}\n")
        f.write(f"NODATA_value {nodata_value!r}\n")
        for row in out:
            f.write(" ".join(fmt % v for v in row))
            f.write("\n")


def read_hydrograph(path: str):
    """Mode-II inflow table: returns (t, Q, phi_s) as float64 arrays (phi_s
    None when the file has two columns).  Times must increase."""
    rows = []
    with open(path) as f:
        for line in f:
            s = line.split("#", 1)[0].strip()
            if s:
                rows.append([float(v) for v in s.replace(",", " ").split()])
    if not rows or len({len(r) for r in rows}) != 1 or len(rows[0]) not in (2, 3):
        raise ValueError(f"{path}: need rows of 2 or 3 numbers (t, Q[, phi_s])")
    a = np.array(rows)
    if np.any(np.diff(a[:, 0]) <= 0):
        raise ValueError(f"{path}: times must increase")
    return a[:, 0].copy(), a[:, 1].copy(), (a[:, 2].copy() if a.shape[1] == 3 else None)


def config_from_asc(dem_path: str, params: dict, h_path: str | None = None, phi_path: str | None = None,
                    phi_s: float = 0.5, inflow: dict | None = None, name: str | None = None) -> dict:
    """A workload dict (the shape `moses.from_config` and the oracle take)
    from .asc files: the DEM, and for Mode I the release thickness h [m]
    (normal to the bed) and optionally its solid fraction (else `phi_s`
    everywhere); for Mode II an `inflow` dict (side, i0, i1, t, Q, phi) as in
    `workloads.inflow_config`.  NODATA in the DEM is an error; in h it reads
    as 0."""
    dem, hd = read_asc(dem_path)
    if not np.isfinite(dem).all():
        raise ValueError(f"{dem_path}: the DEM has NODATA cells; fill them before running")
    shape = dem.shape
    if h_path is not None:
        h, hh = read_asc(h_path, nodata=0.0)
        if h.shape != shape or hh["dx"] != hd["dx"] or hh["dy"] != hd["dy"]:
            raise ValueError(f"{h_path}: grid differs from the DEM's")
    else:
        h = np.zeros(shape)
    if phi_path is not None:
        phi, ph = read_asc(phi_path, nodata=phi_s)
        if phi.shape != shape:
            raise ValueError(f"{phi_path}: grid differs from the DEM's")
    else:
        phi = np.full(shape, float(phi_s))
    cfg = dict(name=name or os.path.basename(dem_path), dem=dem, dx=hd["dx"], dy=hd["dy"], params=dict(params),
               h=h, phi_s=phi, origin=(hd["xll"], hd["yll"]))
    if inflow is not None:
        cfg["inflow"] = dict(inflow)
    return cfg


def write_state_asc(state: dict, prefix: str, dx: float, dy: float | None = None, xll: float = 0.0,
                    yll: float = 0.0):
    """Write the output fields of `Sim.get_state()` (h, phi_s, vx_s, vy_s,
    vx_f, vy_f) as `<prefix>_<field>.asc`; returns the paths."""
    paths = []
    for key in ("h", "phi_s", "vx_s", "vy_s", "vx_f", "vy_f"):
        p = f"{prefix}_{key}.asc"
        write_asc(p, state[key], dx, dy, xll, yll)
        paths.append(p)
    return paths
