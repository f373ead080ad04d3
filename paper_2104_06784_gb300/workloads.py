"""Seeded synthetic inputs: DEMs, release piles, inflow hydrographs, parameter sets.

This module holds no arithmetic of the flow model.  It produces the inputs that
both the CUDA library and the CPU oracle consume, so that the two never share
anything else.  The real terrains of the paper (the 2009 Hsiaolin landslide,
Sect. 4.1, and the DF004 debris flow, Sect. 4.2) are not available; the
generators below stand in for them with the shapes and sizes of those events:
a >2e7 m^3 release at 10 m resolution on steep rugged terrain (Hsiaolin scale)
and a channelised inflow hydrograph at 5 m resolution (DF004 scale).

Array convention: row-major ``[j, i]`` with ``j = 0`` the southern row
(Y increasing northwards) and ``i = 0`` the western column.
"""
from __future__ import annotations

import math

import numpy as np

# ----------------------------------------------------------------------------
# parameter sets (SI).  Keys mirror the moses_params / oracle parameter struct.

BC_CLOSED = 0
BC_TRANSMISSIVE = 1
SIDE_W, SIDE_E, SIDE_S, SIDE_N = 0, 1, 2, 3


def default_params(**over) -> dict:
    """Rheology of the synthetic release configurations (SI units).

    rho_s / rho_f = 2700 / 1100 kg m^-3, basal friction 25 deg, internal friction
    35 deg (only used by the earth-pressure option), drag 1e-3 1/s, no fluid
    viscosity or fluid basal friction (the configurations give no N_R or
    vartheta_b), CFL 0.1 as in Sect. 2.2, thin-layer threshold 1 mm (below it a
    phase carries no velocity).
    """
    p = dict(
        g=9.81,
        eps=1.0,
        eps_chi=1.0,
        rho_s=2700.0,
        rho_f=1100.0,
        delta_b_deg=25.0,
        phi_int_deg=35.0,
        k_mode=0,
        c_d=1e-3,
        nu_f=0.0,
        k_f=0.0,
        cfl=0.1,
        dt_max=1.0,
        h_dry=1e-3,
        bc=(BC_CLOSED,) * 4,
        fluid_pg_mode=0,
        scheme=0,
        recon=0,
        rk=2,
    )
    p.update(over)
    return p


# ----------------------------------------------------------------------------
# DEMs


def flat_dem(nx: int, ny: int) -> np.ndarray:
    return np.zeros((ny, nx))


def incline_dem(nx: int, ny: int, dx: float, dy: float, zeta_deg: float, axis: str = "x") -> np.ndarray:
    """Plane falling towards +X (axis='x') or +Y (axis='y') at angle zeta."""
    t = math.tan(math.radians(zeta_deg))
    if axis == "x":
        x = (np.arange(nx) + 0.5) * dx
        return np.broadcast_to(-t * x[None, :], (ny, nx)).copy()
    y = (np.arange(ny) + 0.5) * dy
    return np.broadcast_to(-t * y[:, None], (ny, nx)).copy()


def arc_plane_dem(nx: int = 128, ny: int = 128, dx: float = 5.0, dy: float = 5.0,
                  y0: float = 200.0, radius: float = 100.0, zeta_deg: float = 35.0) -> np.ndarray:
    """Horizontal runout for Y <= y0, a circular arc of the given radius tangent
    to it, and a plane at zeta_deg above the arc (rising to the north)."""
    y = (np.arange(ny) + 0.5) * dy
    z = math.radians(zeta_deg)
    y1 = y0 + radius * math.sin(z)
    b1 = radius * (1.0 - math.cos(z))
    b = np.where(y <= y0, 0.0,
                 np.where(y <= y1, radius - np.sqrt(np.maximum(radius ** 2 - (y - y0) ** 2, 0.0)),
                          b1 + (y - y1) * math.tan(z)))
    return np.broadcast_to(b[:, None], (ny, nx)).copy()


def paraboloid_dem(nx: int, ny: int, dx: float, dy: float, cxx: float, cxy: float, cyy: float) -> np.ndarray:
    """b = (cxx X^2 + 2 cxy X Y + cyy Y^2) / 2 about the grid centre."""
    x = (np.arange(nx) + 0.5) * dx - nx * dx / 2
    y = (np.arange(ny) + 0.5) * dy - ny * dy / 2
    X, Y = np.meshgrid(x, y)
    return 0.5 * (cxx * X ** 2 + 2 * cxy * X * Y + cyy * Y ** 2)


def spectral_dem(nx: int, ny: int, dx: float, beta: float = 2.2, relief: float = 1500.0,
                 seed: int = 0, band_m: float = 320.0) -> np.ndarray:
    """Seeded 1/f^beta terrain: white noise filtered to a power spectrum
    |k|^-beta (amplitude |k|^-beta/2), rescaled to the given relief.

    The spectrum is rolled off below wavelengths of `band_m` metres (amplitude
    factor exp(-(k band_m)^2)).  Unfiltered, a beta = 2.2 power spectrum puts
    the slopes and the bed curvature at the grid scale: at 4096 x 4096 cells of
    10 m with 1500 m relief the median slope is 76 deg and curvature radii are a
    few metres under tens of metres of flow, outside the shallow ordering of
    the model's equations (the centripetal term of the basal pressure then
    grows with v^2 and the step runs away).  With band_m = 320 m that terrain
    has a median slope of 27 deg, 90th percentile 42 deg, a quarter of the
    cells at 30-40 deg and curvature radii above ~20 m.  band_m = 0 disables
    the roll-off."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((ny, nx))
    W = np.fft.rfft2(w)
    kx = np.fft.rfftfreq(nx, d=dx)
    ky = np.fft.fftfreq(ny, d=dx)
    k = np.sqrt(kx[None, :] ** 2 + ky[:, None] ** 2)
    k[0, 0] = np.inf
    W *= k ** (-beta / 2.0)
    if band_m > 0:
        W *= np.exp(-(np.where(np.isinf(k), 0.0, k) * band_m) ** 2)
    z = np.fft.irfft2(W, s=(ny, nx))
    z -= z.min()
    zmax = z.max()
    return z * (relief / zmax) if zmax > 0 else z


def carve_valley(dem: np.ndarray, dx: float, depth: float = 100.0, half_width: float = 400.0,
                 seed: int = 0) -> np.ndarray:
    """Carve one V-shaped valley along a seeded meander running west-east."""
    ny, nx = dem.shape
    rng = np.random.default_rng(seed + 7919)
    x = (np.arange(nx) + 0.5) * dx
    Ly = ny * dx
    yc = Ly * (0.35 + 0.3 * rng.random())
    amp = Ly * (0.05 + 0.1 * rng.random())
    lam = nx * dx / (1.0 + 2.0 * rng.random())
    ph = 2 * math.pi * rng.random()
    path = yc + amp * np.sin(2 * math.pi * x / lam + ph)
    y = (np.arange(ny) + 0.5) * dx
    d = np.abs(y[:, None] - path[None, :])
    return dem - depth * np.clip(1.0 - d / half_width, 0.0, None)


def channel_fan_dem(nx: int = 2048, ny: int = 1024, dx: float = 5.0, channel_frac: float = 0.4,
                    thalweg_deg: float = 15.0, bank_deg: float = 30.0, fan_deg: float = 5.0,
                    taper: float = 500.0) -> np.ndarray:
    """V-channel along X (thalweg at thalweg_deg, banks at bank_deg) over the
    first channel_frac of the length, opening onto a fan_deg plane whose banks
    fade out over `taper` metres.  Flow runs west to east."""
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dx
    Lc = channel_frac * nx * dx
    yc = ny * dx / 2
    X, Y = np.meshgrid(x, y)
    dY = np.abs(Y - yc)
    bank = math.tan(math.radians(bank_deg)) * dY
    z_apex = math.tan(math.radians(fan_deg)) * (nx * dx - Lc) + 10.0
    ch = z_apex + math.tan(math.radians(thalweg_deg)) * (Lc - X) + bank
    w = np.clip(1.0 - (X - Lc) / taper, 0.0, 1.0)
    fan = z_apex - math.tan(math.radians(fan_deg)) * (X - Lc) + bank * w
    return np.where(X <= Lc, ch, fan)


# ----------------------------------------------------------------------------
# releases and inflow


def parabolic_cap(nx: int, ny: int, dx: float, dy: float, ic: float, jc: float, radius_cells: float,
                  hmax: float) -> np.ndarray:
    """h = hmax (1 - r^2/R^2)_+ with r the horizontal distance to cell (ic, jc)
    and R = radius_cells * dx."""
    x = (np.arange(nx) - ic) * dx
    y = (np.arange(ny) - jc) * dy
    R = radius_cells * dx
    r2 = x[None, :] ** 2 + y[:, None] ** 2
    return hmax * np.clip(1.0 - r2 / R ** 2, 0.0, None)


def triangular_hydrograph(q_peak: float = 800.0, t_peak: float = 60.0, t_end: float = 300.0,
                          phi_s: float = 0.5):
    t = np.array([0.0, t_peak, t_end])
    Q = np.array([0.0, q_peak, 0.0])
    phi = np.full(3, phi_s)
    return t, Q, phi


def release_volume(h: np.ndarray, dem: np.ndarray, dx: float) -> float:
    """Volume of a layer of normal thickness h over the DEM: sum J h dx dy,
    with J = sqrt(1 + b_X^2 + b_Y^2) from central differences of the DEM (the
    area of the bed surface over a cell is J dx dy)."""
    gy, gx = np.gradient(dem, dx)
    return float((h * np.sqrt(1.0 + gx * gx + gy * gy)).sum() * dx * dx)


def slope_deg(dem: np.ndarray, dx: float) -> np.ndarray:
    """Terrain slope angle from numpy's gradient (used only to place releases)."""
    gy, gx = np.gradient(dem, dx)
    return np.degrees(np.arctan(np.hypot(gx, gy)))


# ----------------------------------------------------------------------------
# the configurations (full size, or scaled down with the same structure)


def release_config(nx: int = 128, ny: int = 128, dx: float = 5.0, **over) -> dict:
    """Arc-plane DEM with a parabolic-cap mixture pile (max depth 5 m, radius
    20 cells, centred 30 cells below the top edge), solid fraction 0.6, closed
    boundaries, CFL 0.5, 2000 steps, FP64."""
    dem = arc_plane_dem(nx, ny, dx, dx)
    h = parabolic_cap(nx, ny, dx, dx, nx // 2, ny - 1 - 30 * ny // 128, 20 * nx / 128, 5.0)
    phi = np.full((ny, nx), 0.6)
    p = default_params(cfl=0.5, bc=(BC_CLOSED,) * 4)
    p.update(over)
    return dict(name=f"arc-plane release {nx}x{ny} dx={dx} m", dem=dem, dx=dx, dy=dx, params=p, h=h,
                phi_s=phi, steps=2000)


def large_release_config(n: int = 4096, dx: float = 10.0, seed: int = 0, ny: int | None = None,
                         volume: float = 2.5e7, radius_cells: float = 43.0, **over) -> dict:
    """Spectral 1/f^2.2 DEM (1500 m relief) with one carved valley; a 2.5e7 m^3
    parabolic-cap release of radius 43 cells centred on the seeded cell whose
    slope is nearest 35 deg within 30-40 deg (the volume counted normal to the
    bed, sum J h dx dy); solid fraction U(0.55, 0.65) per cell; transmissive
    boundaries; CFL 0.1; 10000 steps."""
    ny = ny or n
    nx = n
    relief = 1500.0 * min(1.0, max(nx, ny) / 4096.0) if (nx < 4096) else 1500.0
    dem = spectral_dem(nx, ny, dx, 2.2, relief, seed)
    dem = carve_valley(dem, dx, depth=100.0 * relief / 1500.0, half_width=40 * dx, seed=seed)
    rng = np.random.default_rng(seed + 104729)
    sl = slope_deg(dem, dx)
    m = int(math.ceil(radius_cells)) + 2
    inner = np.zeros_like(sl, dtype=bool)
    if nx > 2 * m and ny > 2 * m:
        inner[m:ny - m, m:nx - m] = True
    else:
        inner[:, :] = True
    band = inner & (sl >= 30.0) & (sl <= 40.0)
    cand = np.argwhere(band) if band.any() else np.argwhere(inner)
    score = np.abs(sl[cand[:, 0], cand[:, 1]] - 35.0) + 1e-3 * rng.random(len(cand))
    jc, ic = cand[int(np.argmin(score))]
    shape = parabolic_cap(nx, ny, dx, dx, ic, jc, radius_cells, 1.0)
    h = shape * (volume / release_volume(shape, dem, dx))
    phi = rng.uniform(0.55, 0.65, size=(ny, nx))
    p = default_params(cfl=0.1, bc=(BC_TRANSMISSIVE,) * 4)
    p.update(over)
    return dict(name=f"spectral-DEM release {nx}x{ny} dx={dx} m", dem=dem, dx=dx, dy=dx, params=p, h=h,
                phi_s=phi, steps=10000, release_cell=(int(ic), int(jc)))


def adjoint_config(n: int = 1024, dx: float = 5.0, seed: int = 0, **over) -> dict:
    """Calibration workload: the large-release terrain at n x n cells of dx
    (spectral DEM, relief 1500 m x n / 4096, one carved valley) with a
    1e6 m^3 parabolic-cap release of radius 43 cells on a 30-40 deg slope;
    internal friction 35 deg through the Savage-Hutter earth-pressure option
    (k_mode 1), so that both friction angles have gradients; FP32 state; 5000
    steps with a checkpoint every 71; the target deposit comes from the hidden
    basal friction 22 deg and drag 3e-3 1/s, the start is 25 deg and
    1e-3 1/s."""
    over = dict(dict(k_mode=1), **over)
    cfg = large_release_config(n=n, dx=dx, seed=seed, volume=1e6, radius_cells=43.0, **over)
    cfg.update(name=f"adjoint calibration {n}x{n} dx={dx} m", steps=5000, ckpt_every=71, precision="fp32",
               hidden=dict(delta_b_deg=22.0, c_d=3e-3))
    return cfg


def inflow_config(nx: int = 2048, ny: int = 1024, dx: float = 5.0, inlet_cells: int = 20, **over) -> dict:
    """Channel-and-fan DEM with a triangular hydrograph (peak 800 m^3/s at
    60 s, zero by 300 s, solid fraction 0.5) at an inlet of `inlet_cells`
    cells on the west edge centred on the thalweg; transmissive elsewhere;
    simulated to 600 s; FP32 state with FP64 budgets."""
    dem = channel_fan_dem(nx, ny, dx)
    t, Q, phi = triangular_hydrograph()
    j0 = ny // 2 - inlet_cells // 2
    p = default_params(cfl=0.1, bc=(BC_TRANSMISSIVE,) * 4)
    p.update(over)
    return dict(name=f"channel-fan inflow {nx}x{ny} dx={dx} m", dem=dem, dx=dx, dy=dx, params=p,
                h=np.zeros((ny, nx)), phi_s=np.zeros((ny, nx)),
                inflow=dict(side=SIDE_W, i0=j0, i1=j0 + inlet_cells, t=t, Q=Q, phi=phi),
                t_end=600.0)


def ensemble_sides(n: int = 256, seed: int = 0, lo: int = 64, hi: int = 1024) -> list[int]:
    """Grid sides: clip(round16(exp(N(ln 256, (ln 4 / 2)^2))), 64, 1024)."""
    rng = np.random.default_rng(seed)
    z = np.exp(rng.normal(math.log(256.0), math.log(4.0) / 2.0, size=n))
    return [int(min(hi, max(lo, 16 * round(v / 16.0)))) for v in z]


def ensemble_config(n: int = 256, seed: int = 0, dx: float = 5.0, lo: int = 64, hi: int = 1024) -> list[dict]:
    """Independent scenarios on uneven square grids: each a seeded spectral
    DEM (beta 2.2, relief 0.15 N dx, rolled off below 320 m wavelength like
    the large-release terrain: median slopes 14-29 deg, 90th percentiles
    21-46 deg from the smallest to the largest grid), basal friction U(15, 30)
    deg, drag U(1e-4, 1e-2) 1/s, release volume U(1e4, 1e6) m^3 (normal to
    the bed, sum J h dx dy) as a parabolic cap at the grid centre whose radius
    is N/16 cells or, for a large volume on a small grid, the radius of a cap
    30 m high (at most N/3 cells), 3000 steps, FP32.  (Steeper terrain --
    relief 0.3 N dx with an 80 m roll-off, median slopes up to 70 deg and bed
    curvature up to 0.4 / m -- and radius N/16 throughout, which piles 1e6 m^3
    into a tower a kilometre high on a 64 x 64 grid, put thin fluid films in
    gullies with 60-70 deg walls, where the step runs away.)"""
    rng = np.random.default_rng(seed + 31337)
    out = []
    for k, N in enumerate(ensemble_sides(n, seed, lo, hi)):
        dem = spectral_dem(N, N, dx, 2.2, 0.15 * N * dx, seed * 100003 + k, band_m=320.0)
        d_b = rng.uniform(15.0, 30.0)
        c_d = rng.uniform(1e-4, 1e-2)
        V = rng.uniform(1e4, 1e6)
        r30 = math.sqrt(2.0 * V / (math.pi * 30.0)) / dx
        shape = parabolic_cap(N, N, dx, dx, N // 2, N // 2, min(max(N / 16.0, r30), N / 3.0), 1.0)
        h = shape * (V / release_volume(shape, dem, dx))
        p = default_params(delta_b_deg=d_b, c_d=c_d, cfl=0.1, bc=(BC_TRANSMISSIVE,) * 4)
        out.append(dict(name=f"ensemble member {k} ({N}x{N})", dem=dem, dx=dx, dy=dx, params=p, h=h,
                        phi_s=np.full((N, N), 0.6), steps=3000))
    return out


def random_state(nx: int, ny: int, seed: int = 0, depth: float = 2.0, speed: float = 3.0,
                 dry_frac: float = 0.2) -> dict:
    """A rough random flow state (normal thickness, solid fraction, phase
    velocities) with dry patches, for single-stage parity checks."""
    rng = np.random.default_rng(seed)
    h = depth * rng.random((ny, nx))
    h[rng.random((ny, nx)) < dry_frac] = 0.0
    return dict(h=h, phi_s=rng.uniform(0.3, 0.8, (ny, nx)),
                vx_s=speed * rng.standard_normal((ny, nx)), vy_s=speed * rng.standard_normal((ny, nx)),
                vx_f=speed * rng.standard_normal((ny, nx)), vy_f=speed * rng.standard_normal((ny, nx)))
