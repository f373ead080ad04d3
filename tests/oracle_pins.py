"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each ``pin_*`` function builds small seeded inputs, runs the oracle (the default
build, or a build with a planted mistake passed as ``L``) and raises
``AssertionError`` when the oracle departs from a closed form, an invariant, a
textbook special case or an exact identity.  None of them retypes an oracle
formula.  They compare the oracle with:
- analytic solutions (Ritter, Savage-Hutter);
- conservation laws and symmetries (rotation, mirror, the solid and fluid
  phases);
- differential-geometric identities;
- the schemes' own definitions of a step from its stages.
Each is chosen so that a plausible mistake in the part it covers fails it:
``tests/test_oracle_mutants.py`` plants such mistakes.

Citations are to arXiv:2104.06784 (App. A equations by label, Sect. 2.1-2.2).
"""
from __future__ import annotations

import math

import numpy as np

from oracle.oracle import OracleSim
from paper_2104_06784_gb300 import workloads as W

G = 9.81


def _sim(dem, dx, dy, params, L):
    return OracleSim(dem, dx, dy, params, library=L)


def _pure_fluid(**over):
    return W.default_params(**over)


def _pure_solid(**over):
    p = W.default_params(rho_f=0.0, **over)  # alpha_rho = 0
    return p


# ----------------------------------------------------------------------------
# geometry (Sect. 2.1; App. A: J_b = det Omega_b, (A_ij) = Omega_b^-1, n, c = n_Z)


def pin_geometry_plane(L=None):
    """Inclined planes: J = sec(zeta), c = cos(zeta), n = (sin z cos t,
    sin z sin t, cos z), the 2x2 block of Omega_b^-1 inverts the surface metric
    g = I + grad b grad b^T, dn = 0, and v_xi = v_X, v_eta = v_Y."""
    nx, ny, dx = 12, 10, 3.0
    for zeta in (0.0, 20.0, 35.0, 60.0):
        for theta in (0.0, 37.0, 90.0, 200.0):
            tz, th = math.radians(zeta), math.radians(theta)
            x = (np.arange(nx) + 0.5) * dx
            y = (np.arange(ny) + 0.5) * dx
            X, Y = np.meshgrid(x, y)
            dem = -math.tan(tz) * (X * math.cos(th) + Y * math.sin(th))
            s = _sim(dem, dx, dx, W.default_params(), L)
            g = s.geometry()
            tol = 1e-12
            assert np.allclose(g["J"], 1 / math.cos(tz), rtol=tol, atol=0), "J_b != sec(zeta)"
            assert np.allclose(g["c"], math.cos(tz), rtol=tol, atol=tol), "c != cos(zeta)"
            n_ex = (math.sin(tz) * math.cos(th), math.sin(tz) * math.sin(th), math.cos(tz))
            for k, name in enumerate(("nX", "nY", "nZ")):
                assert np.allclose(g[name], n_ex[k], atol=tol), f"{name} wrong"
            bx = -math.tan(tz) * math.cos(th)
            by = -math.tan(tz) * math.sin(th)
            gm = np.array([[1 + bx * bx, bx * by], [bx * by, 1 + by * by]])
            A = np.array([[g["A11"][3, 4], g["A12"][3, 4]], [g["A21"][3, 4], g["A22"][3, 4]]])
            assert np.allclose(A @ gm, np.eye(2), atol=1e-12), "A is not the inverse metric"
            for name in ("dnX_dxi", "dnY_dxi", "dnZ_dxi", "dnX_deta", "dnY_deta", "dnZ_deta"):
                assert np.abs(g[name]).max() < 1e-12, f"{name} != 0 on a plane"
            vx, vy = 1.7, -0.6
            xi, eta = s.tangential(4, 3, vx, vy)
            assert abs(xi - vx) < 1e-13 and abs(eta - vy) < 1e-13, "v_xi != v_X under xi = X"
    # the incline along X: A = diag(cos^2 zeta, 1)
    s = _sim(W.incline_dem(8, 6, 2.0, 2.0, 30.0), 2.0, 2.0, W.default_params(), L)
    g = s.geometry()
    assert np.allclose(g["A11"], math.cos(math.radians(30)) ** 2, atol=1e-14)
    assert np.allclose(g["A22"], 1.0, atol=1e-14)


def pin_curvature(L=None):
    """kappa (App. A, below Eq. Src_nd_Topo) is the normal curvature times the
    squared 3D speed, negative on a concave bed: on a quadratic surface it
    equals -II(v, v)/|m| exactly; on the arc of radius R it tends to -V^2/R."""
    # quadratic surface: second differences are exact there
    nx, ny, dx = 20, 18, 4.0
    cxx, cxy, cyy = 0.004, -0.0015, 0.0025
    dem = W.paraboloid_dem(nx, ny, dx, dx, cxx, cxy, cyy)
    s = _sim(dem, dx, dx, W.default_params(), L)
    x = (np.arange(nx) + 0.5) * dx - nx * dx / 2
    y = (np.arange(ny) + 0.5) * dx - ny * dx / 2
    for (i, j) in ((3, 4), (10, 9), (16, 2)):
        bX = cxx * x[i] + cxy * y[j]
        bY = cxy * x[i] + cyy * y[j]
        for (vx, vy) in ((2.0, 0.0), (-1.0, 3.0), (0.7, -2.2)):
            ex = -(cxx * vx * vx + 2 * cxy * vx * vy + cyy * vy * vy) / math.sqrt(1 + bX * bX + bY * bY)
            got = s.kappa(i, j, vx, vy)
            assert abs(got - ex) <= 1e-12 * (abs(ex) + 1e-12), f"kappa {got} != {ex} on a paraboloid"
    # a unit normal's derivatives are orthogonal to it: n . dn/dxi = n . dn/deta = 0
    g = s.geometry()
    for d in ("dxi", "deta"):
        dot = g["nX"] * g[f"dnX_{d}"] + g["nY"] * g[f"dnY_{d}"] + g["nZ"] * g[f"dnZ_{d}"]
        assert np.abs(dot).max() < 1e-15, f"n . dn/{d} != 0"
    # circular arc (radius 100 m): kappa -> -V^2/R with O(dy^2) error
    errs = []
    for dy in (2.0, 1.0):
        ny = int(400 / dy)
        dem = W.arc_plane_dem(4, ny, dy, dy)
        s = _sim(dem, dy, dy, W.default_params(), L)
        y = (np.arange(ny) + 0.5) * dy
        j = int(np.argmin(np.abs(y - 228.0)))  # inside the arc (200 .. 257 m)
        by = (y[j] - 200.0) / math.sqrt(100.0 ** 2 - (y[j] - 200.0) ** 2)
        vy = 5.0
        V2 = vy * vy * (1 + by * by)
        errs.append(abs(s.kappa(1, j, 0.0, vy) + V2 / 100.0) / (V2 / 100.0))
    assert errs[-1] < 1e-3, f"arc curvature error {errs[-1]}"
    assert errs[0] / max(errs[1], 1e-300) > 3.0, f"arc curvature not second order: {errs}"


# ----------------------------------------------------------------------------
# conservation (Eqs. MassEq_TopoS0/F0) with closed boundaries


def pin_conservation_closed(L=None, steps=300):
    cfg = W.release_config(cfl=0.1)
    s = _sim(cfg["dem"], cfg["dx"], cfg["dy"], cfg["params"], L)
    s.set_release(cfg["h"], cfg["phi_s"])
    b0 = s.budget()
    s.step(steps)
    b = s.budget()
    assert b["clamp_cells"] == 0, "positivity clamp fired at CFL 0.1"
    for ph in ("s", "f"):
        rel = abs(b[f"vol_{ph}"] - b0[f"vol_{ph}"]) / b0[f"vol_{ph}"]
        assert rel < 1e-13, f"phase {ph} volume drift {rel}"
    # symmetric pile on an X-invariant bed: no net X momentum
    assert abs(b["mom_xs"]) < 1e-9 * abs(b["mom_ys"]) and abs(b["mom_xf"]) < 1e-9 * abs(b["mom_yf"])
    assert b["mom_ys"] < 0 and b["mom_yf"] < 0, "pile does not move downslope (south)"


# ----------------------------------------------------------------------------
# bodies at rest


def pin_lake_flat(L=None):
    nx = ny = 16
    s = _sim(W.flat_dem(nx, ny), 5.0, 5.0, _pure_fluid(), L)
    s.set_release(np.full((ny, nx), 2.0), np.zeros((ny, nx)))
    U0 = s.get_U()
    s.step(20)
    U = s.get_U()
    assert np.abs(U[[1, 2, 4, 5]]).max() == 0.0, "flat lake moved"
    assert np.abs(U - U0).max() < 1e-14


def _plane_equilibrium(L, phi_s, delta_b, zeta=20.0, fluid_pg_mode=0, eps=1.0):
    """Depth with dh/dX = sin(zeta)/(eps cos^2(zeta)): the leading-order
    model's own hydrostatic state of a fluid on a plane (dh/ds = tan(zeta)
    along slope for eps = 1).  At rest the fluid's X-momentum balance is
    eps d(J h A_11 g c h / 2)/dX = J g c h |n_X|: the pressure flux carries
    eps, the basal normal source does not, and A_11 = cos^2(zeta), |n_X| =
    sin(zeta).  Returns the largest interior momentum after two steps and its
    scale."""
    nx, ny, dx, dt = 64, 5, 2.0, 0.05
    dem = W.incline_dem(nx, ny, dx, dx, zeta)
    tz = math.radians(zeta)
    x = (np.arange(nx) + 0.5) * dx
    h = np.broadcast_to(2.0 + x * math.sin(tz) / (eps * math.cos(tz) ** 2), (ny, nx)).copy()
    p = W.default_params(delta_b_deg=delta_b, bc=(W.BC_TRANSMISSIVE,) * 4, fluid_pg_mode=fluid_pg_mode, eps=eps)
    s = _sim(dem, dx, dx, p, L)
    s.set_release(h, np.full((ny, nx), phi_s))
    s.step_dt(dt)
    s.step_dt(dt)
    U = s.get_U()
    inner = U[:, :, 12:nx - 12]
    scale = dt * G * h.max() * math.sin(tz) * (1 / math.cos(tz))
    return max(np.abs(inner[[1, 2, 4, 5]]).max(), 0.0), scale


def pin_lake_plane(L=None):
    m, scale = _plane_equilibrium(L, phi_s=0.0, delta_b=25.0)
    assert m < 1e-12 * scale, f"fluid equilibrium on a plane moved: {m}"


def _curved_lake_residual(L, nx, A=20.0, Lx=800.0, C0=25.0):
    """The model's own fluid state at rest on a bed b(X) curved along X only:
    with c = n_Z = (1 + b'^2)^(-1/2), J = 1/c and A_11 = c^2 the X-momentum
    balance at rest eps d(J h A_11 g c h / 2)/dX = J g c h |n_X| becomes
    eps d(c h)/dX = -b'(X), so c h + b / eps is constant (the plane case of
    _plane_equilibrium is the special case of constant c).  On b = A cos(2 pi X
    / Lx) with c h = C0 - b (eps = 1) one step of size 0.25 dx / sqrt(g h_max)
    is taken; returns the largest and the mean fluid X-momentum of the middle
    70 % of the span, each over dt g h_max max|b'| (the residual force of the
    discrete scheme, which is not well-balanced on curved beds)."""
    ny = 5
    dx = Lx / nx
    x = (np.arange(nx) + 0.5) * dx
    b1 = A * np.cos(2 * math.pi * x / Lx)
    bp = -A * 2 * math.pi / Lx * np.sin(2 * math.pi * x / Lx)
    c = 1.0 / np.sqrt(1.0 + bp ** 2)
    h = np.broadcast_to((C0 - b1) / c, (ny, nx)).copy()
    dem = np.broadcast_to(b1, (ny, nx)).copy()
    p = W.default_params(delta_b_deg=25.0, bc=(W.BC_TRANSMISSIVE,) * 4)
    s = _sim(dem, dx, dx, p, L)
    s.set_release(h, np.zeros((ny, nx)))
    dt = 0.25 * dx / math.sqrt(G * h.max())
    s.step_dt(dt)
    U = s.get_U()
    a, b = int(0.15 * nx), int(0.85 * nx)
    r = np.abs(U[4, ny // 2, a:b]) / (dt * G * h.max() * np.abs(bp).max())
    return r.max(), r.mean()


def pin_lake_curved_bed_residual_converges(L=None):
    """The fluid at rest on a cosine bed (c h + b constant, see
    _curved_lake_residual) is not an exact discrete equilibrium of the central
    scheme (Sect. 2.2 has no well-balanced reconstruction), but its residual
    force converges: the mean at second order, the largest (at the trough,
    where minmod clips the depth's extremum) at first order, over 64, 128 and
    256 cells; a sign error or a dropped geometry factor in the pressure flux
    or the basal source leaves an O(1) residual that does not converge."""
    res = [_curved_lake_residual(L, nx) for nx in (64, 128, 256)]
    for (m0, a0), (m1, a1) in zip(res, res[1:]):
        assert m0 / m1 > 1.8, f"largest residual not first order: {m0} -> {m1}"
        assert a0 / a1 > 3.5, f"mean residual not second order: {a0} -> {a1}"
    assert res[-1][0] < 6e-3 and res[-1][1] < 2e-4, res[-1]


def pin_plane_equilibrium_eps(L=None):
    """The plane equilibria of pin_lake_plane and pin_mixture_plane_rest with
    the aspect ratio eps of the dimensionless equations (App. A) other than
    1: the equilibrium slope of the depth scales as 1/eps, and a mixture stays
    at rest only if the fluid's pressure-gradient source carries the same eps
    as the pressure flux (Eq. SrcF_f_Topo)."""
    for eps in (0.5, 2.0):
        for phi_s, delta_b in ((0.0, 25.0), (0.6, 35.0)):
            m, scale = _plane_equilibrium(L, phi_s=phi_s, delta_b=delta_b, eps=eps)
            assert m < 1e-12 * scale, f"plane equilibrium with eps = {eps}, phi_s = {phi_s} moved: {m}"


def pin_mixture_plane_rest(L=None):
    """Mixture (phi^s = 0.6) in the fluid's equilibrium on a 20 deg plane with
    basal friction strong enough to hold the grains: stays at rest only if the
    fluid feels -phi^f grad P overall, i.e. the pressure-gradient source of the
    fluid carries phi^s (reading R1 of Eq. SrcF_f_Topo)."""
    m, scale = _plane_equilibrium(L, phi_s=0.6, delta_b=25.0)
    assert m < 1e-12 * scale, f"mixture equilibrium on a plane moved: {m}"


def pin_heap_rest(L=None):
    """Pure-solid parabolic heap (surface slope 0.1 < tan 25 deg) on a flat bed
    and on a 20 deg plane: every cell of the heap stays exactly at rest
    (Coulomb stopping, Eq. Src_nd_Topo).  The central scheme's numerical
    diffusion wets the margin, where the neighbour's face pressure pushes cells
    whose friction was zero at the stage start; that creep must die out (Heun
    halves a stopped cell's momentum each step).  On a 30 deg plane the heap
    slides (sin 30 > cos 30 tan 25)."""
    nx = ny = 48
    dx = 5.0
    h = W.parabolic_cap(nx, ny, dx, dx, 24, 24, 20, 5.0)
    heap = h > 0
    for dem, moves in ((W.flat_dem(nx, ny), False), (W.incline_dem(nx, ny, dx, dx, 20.0), False),
                       (W.incline_dem(nx, ny, dx, dx, 30.0), True)):
        s = _sim(dem, dx, dx, _pure_solid(delta_b_deg=25.0), L)
        s.set_release(h, np.ones((ny, nx)))
        s.step(30)
        U = s.get_U()
        mom = np.abs(U[1:3]).max(axis=0)
        if moves:
            assert mom[heap].max() > 1e-2, "heap held on a 30 deg plane with a 25 deg friction angle"
            continue
        assert mom[heap].max() == 0.0, f"heap at rest moved ({mom[heap].max()})"
        s.step(70)
        pr = s.primitive()
        assert np.abs(s.get_U()[1:3])[:, heap].max() == 0.0, "heap at rest moved"
        vmax = max(np.abs(pr[k]).max() for k in ("vx_s", "vy_s"))
        assert vmax < 1e-15, f"margin creep does not die out ({vmax} m/s)"


# ----------------------------------------------------------------------------
# Ritter dam break: pure fluid, flat, frictionless (exact shallow-water solution)


def _ritter_error(L, dx, t_end=20.0, h0=10.0, length=2000.0, scheme=0, recon=0, rk=2, want_max=False):
    nx = int(length / dx)
    x = (np.arange(nx) + 0.5) * dx - length / 2
    h = np.where(x < 0, h0, 0.0)[None, :]
    s = _sim(W.flat_dem(nx, 1), dx, dx, _pure_fluid(cfl=0.1, scheme=scheme, recon=recon, rk=rk), L)
    s.set_release(h, np.zeros((1, nx)))
    steps = 0
    while s.t < t_end:
        s.step(10)
        steps += 10
        if steps > 40 * nx:  # the time step collapsed (a broken scheme): fail, do not hang
            return (math.inf, math.inf) if want_max else math.inf
    t = s.t
    c0 = math.sqrt(G * h0)
    ex = np.where(x < -c0 * t, h0, np.where(x > 2 * c0 * t, 0.0, (2 * c0 - x / t) ** 2 / (9 * G)))
    num = s.primitive()["h"][0]
    err = np.abs(num - ex).sum() / ex.sum()
    return (err, num.max()) if want_max else err


def pin_ritter(L=None):
    e10 = _ritter_error(L, 10.0)
    e5 = _ritter_error(L, 5.0)
    assert e5 < 0.01, f"Ritter L1 error {e5} at 400 cells"
    assert e5 < 0.75 * e10, f"Ritter error does not converge: {e10} -> {e5}"


# ----------------------------------------------------------------------------
# Savage-Hutter similarity solution (pure solid, K = 1, plane at zeta)


def _sh_reference(t_end, H0, L0, zeta, delta):
    """Centre s_c and half-length L of the parabolic cap: s_c'' = g (sin z -
    tan d cos z), L'' = 2 g cos z H0 L0 / L^2 (RK4, fine steps)."""
    a = G * (math.sin(zeta) - math.tan(delta) * math.cos(zeta))
    k = 2 * G * math.cos(zeta) * H0 * L0

    def f(y):
        return np.array([y[1], k / y[0] ** 2])

    y = np.array([L0, 0.0])
    n = 20000
    h = t_end / n
    for _ in range(n):
        k1 = f(y)
        k2 = f(y + 0.5 * h * k1)
        k3 = f(y + 0.5 * h * k2)
        k4 = f(y + h * k3)
        y = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return 0.5 * a * t_end ** 2, y[0]


def pin_savage_hutter(L=None):
    zeta, delta = math.radians(35.0), math.radians(25.0)
    H0, L0, dx = 5.0, 100.0, 1.0
    nx = 1400
    x = (np.arange(nx) + 0.5) * dx
    X0 = 200.0
    h = H0 * np.clip(1 - ((x - X0) / (L0 * math.cos(zeta))) ** 2, 0, None)
    s = _sim(W.incline_dem(nx, 1, dx, dx, 35.0), dx, dx, _pure_solid(delta_b_deg=25.0, cfl=0.1), L)
    s.set_release(h[None, :], np.ones((1, nx)))
    t_end = 8.0
    while s.t < t_end:
        s.step(5)
    ds_ref, L_ref = _sh_reference(s.t, H0, L0, zeta, delta)
    U1 = s.get_U()[0, 0]
    sc = x / math.cos(zeta)  # arc length along the slope
    m = U1.sum()
    c = (sc * U1).sum() / m
    var = ((sc - c) ** 2 * U1).sum() / m
    ds = c - X0 / math.cos(zeta)
    Lnum = math.sqrt(5 * var)  # parabola: variance = L^2 / 5
    assert abs(ds - ds_ref) / ds_ref < 5e-3, f"SH centre travel {ds} vs {ds_ref}"
    assert abs(Lnum - L_ref) / (L_ref - L0) < 0.05, f"SH half-length {Lnum} vs {L_ref}"


# ----------------------------------------------------------------------------
# interphase drag (Eqs. Src_v_Topo, SrcF_v_Topo)


def pin_drag(L=None):
    """Uniform mixture on a flat, frictionless bed: rho^s q^s + rho^f q^f is
    conserved, and v^f - v^s decays by the Heun factor 1 - z + z^2/2 per step
    with z = c_D (phi^s + alpha phi^f) dt."""
    nx = ny = 6
    cd, dt, phs = 0.8, 0.1, 0.6
    p = W.default_params(c_d=cd, delta_b_deg=0.0, bc=(W.BC_TRANSMISSIVE,) * 4)
    s = _sim(W.flat_dem(nx, ny), 5.0, 5.0, p, L)
    one = np.ones((ny, nx))
    s.set_release(2.0 * one, phs * one, 1.0 * one, 0.5 * one, 3.0 * one, -1.0 * one)
    al = p["rho_f"] / p["rho_s"]
    z = cd * (phs + al * (1 - phs)) * dt
    U0 = s.get_U()
    mix0 = p["rho_s"] * U0[1:3] + p["rho_f"] * U0[4:6]
    n = 12
    for _ in range(n):
        s.step_dt(dt)
    pr = s.primitive()
    fac = (1 - z + z * z / 2) ** n
    for comp, d0 in (("x", 2.0), ("y", -1.5)):
        dv = pr[f"v{comp}_f"] - pr[f"v{comp}_s"]
        assert np.allclose(dv, d0 * fac, rtol=1e-12, atol=0), f"drag decay {dv.flat[0]} vs {d0 * fac}"
    U = s.get_U()
    mix = p["rho_s"] * U[1:3] + p["rho_f"] * U[4:6]
    assert np.allclose(mix, mix0, rtol=1e-13, atol=1e-12 * np.abs(mix0).max()), "drag not momentum-neutral"


def pin_drag_neutral_on_a_slope(L=None):
    """On a 25-degree plane (J = sec 25 deg, not 1), a uniform mixture with
    different phase velocities, transmissive sides and no basal friction: the
    interphase drag (Eqs. Src_v_Topo, SrcF_v_Topo) moves momentum between the
    phases and adds none to the mixture, so rho^s q^s + rho^f q^f after ten
    steps is the same with the drag as without it, while the phases' own
    momenta differ."""
    nx, ny = 6, 5
    dem = W.incline_dem(nx, ny, 5.0, 4.0, 25.0, "x")
    one = np.ones((ny, nx))
    runs = []
    for cd in (0.0, 0.8):
        p = W.default_params(c_d=cd, delta_b_deg=0.0, bc=(W.BC_TRANSMISSIVE,) * 4)
        s = _sim(dem, 5.0, 4.0, p, L)
        s.set_release(2.0 * one, 0.6 * one, 1.0 * one, 0.5 * one, 3.0 * one, -1.0 * one)
        for _ in range(10):
            s.step_dt(0.05)
        U = s.get_U()
        runs.append((p["rho_s"] * U[1:3] + p["rho_f"] * U[4:6], U[1:3].copy()))
    (m0, q0), (m1, q1) = runs
    assert np.abs(q1 - q0).max() > 1e-3 * np.abs(q0).max(), "the drag changed nothing"
    assert np.allclose(m1, m0, rtol=1e-12, atol=1e-12 * np.abs(m0).max()), "drag not momentum-neutral on a slope"


# ----------------------------------------------------------------------------
# wave speeds and the CFL time step (Sect. 2.2; reading R7)


def pin_wave_speed(L=None):
    """At rest: shallow-water celerity sqrt(g h) for a pure fluid and for a
    pure solid without buoyancy (K = 1); on an X-incline sqrt(g cos z h) across
    the slope; moving fluid adds |v|; dt = CFL min(dx, dy) / a_max."""
    nx, ny = 5, 4
    one = np.ones((ny, nx))
    s = _sim(W.flat_dem(nx, ny), 5.0, 4.0, _pure_fluid(cfl=0.1), L)
    s.set_release(2.0 * one, 0 * one)
    assert abs(s.max_speed() - math.sqrt(G * 2.0)) < 1e-14
    assert abs(s.cfl_dt() - 0.1 * 4.0 / math.sqrt(G * 2.0)) < 1e-15
    s = _sim(W.flat_dem(nx, ny), 5.0, 5.0, _pure_solid(), L)
    s.set_release(3.0 * one, one)
    assert abs(s.max_speed() - math.sqrt(G * 3.0)) < 1e-14
    s = _sim(W.incline_dem(nx, ny, 5.0, 5.0, 30.0), 5.0, 5.0, _pure_fluid(), L)
    s.set_release(2.0 * one, 0 * one)
    assert abs(s.max_speed() - math.sqrt(G * math.cos(math.radians(30)) * 2.0)) < 1e-13
    s = _sim(W.flat_dem(nx, ny), 5.0, 5.0, _pure_fluid(), L)
    s.set_release(2.0 * one, 0 * one, None, None, -3.0 * one, 1.0 * one)
    assert abs(s.max_speed() - (3.0 + math.sqrt(G * 2.0))) < 1e-13
    s = _sim(W.flat_dem(nx, ny), 5.0, 5.0, _pure_fluid(dt_max=0.7), L)
    s.set_release(0 * one, 0 * one)
    assert s.max_speed() == 0.0 and s.cfl_dt() == 0.7, "dry domain must take dt_max"


# ----------------------------------------------------------------------------
# 90 degree rotation invariance


def _rot(f):
    """(X, Y) -> (L - Y, X) on a square grid: f'[j', i'] = f[n - 1 - i', j']."""
    return np.ascontiguousarray(f[::-1, :].T)


def pin_rotation(L=None, steps=40):
    n = 40
    cfg = W.release_config(nx=n, ny=n, cfl=0.2)
    rng = np.random.default_rng(3)
    phi = rng.uniform(0.4, 0.7, (n, n))
    h = cfg["h"] * (1 + 0.2 * rng.random((n, n)))
    dem = cfg["dem"] + rng.random((n, n))
    a = _sim(dem, 5.0, 5.0, cfg["params"], L)
    a.set_release(h, phi)
    b = _sim(_rot(dem), 5.0, 5.0, cfg["params"], L)
    b.set_release(_rot(h), _rot(phi))
    for _ in range(steps):
        dt = a.cfl_dt()
        dtb = b.cfl_dt()
        assert abs(dt - dtb) <= 1e-14 * dt, "rotated run takes a different dt"
        a.step_dt(dt)
        b.step_dt(dt)
    Ua, Ub = a.get_U(), b.get_U()
    exp = np.stack([_rot(Ua[0]), -_rot(Ua[2]), _rot(Ua[1]), _rot(Ua[3]), -_rot(Ua[5]), _rot(Ua[4])])
    scale = np.abs(Ua).max()
    err = np.abs(Ub - exp).max() / scale
    assert err < 1e-12, f"rotation invariance broken: {err}"


# ----------------------------------------------------------------------------
# Mode-II inflow (Sect. 3.1.2; reading R11) and budgets


def pin_inflow(L=None):
    """The ghost state carries the unit discharge Q/W at critical depth
    (v_n equals the model's celerity sqrt(g c A_nn h)); the volume balance
    closes: volume(t) = time-integrated boundary flux + clamp volume."""
    cfg = W.inflow_config(nx=64, ny=40, dx=5.0, inlet_cells=8)
    s = _sim(cfg["dem"], cfg["dx"], cfg["dy"], cfg["params"], L)
    f = cfg["inflow"]
    s.set_inflow(f["side"], f["i0"], f["i1"], f["t"], f["Q"], f["phi"])
    for tt in (30.0, 60.0, 150.0):
        Q = np.interp(tt, f["t"], f["Q"])
        q = Q / ((f["i1"] - f["i0"]) * cfg["dy"])
        for gi in (-1, -2):
            u = s.inflow_state(0, gi, f["i0"] + 2, tt)
            gm = s.cell_geom(gi, f["i0"] + 2)
            Jh = u[0] + u[3]
            vn = (u[1] + u[4]) / Jh
            assert abs(Jh * vn - q) < 1e-12 * q, "inflow ghost does not carry Q/W"
            h = Jh / gm["J"]
            cel = math.sqrt(G * gm["c"] * gm["A11"] * h)
            assert abs(vn - cel) < 1e-12 * cel, "inflow ghost is not at critical depth"
            assert abs(u[0] / Jh - 0.5) < 1e-15
    assert np.all(s.inflow_state(0, -1, f["i0"], 400.0) == 0.0), "no inflow after the hydrograph ends"
    while s.t < 40.0:
        s.step(20)
    b = s.budget()
    for ph in ("s", "f"):
        vol = b[f"vol_{ph}"]
        assert vol > 0
        assert abs(vol - b[f"bnd_in_{ph}"] - b[f"clamp_{ph}"]) < 1e-12 * vol, "volume budget does not close"



def pin_inflow_every_side(L=None):
    """Mode-II inflow (Sect. 3.1.2; R11) on each of the four sides, with cells
    of different width and height and a solid fraction other than 1/2: the
    ghost state splits the mixture as the hydrograph's phi^s at that time
    (linear between its points; no inflow outside its time span), carries the unit
    discharge Q/W (W the segment's length along its side), moves into the
    domain at the model's celerity sqrt(g c A_nn h) (critical depth) and has
    no tangential momentum; over the first steps the volume budget closes:
    volume = time-integrated boundary flux + clamp volume."""
    nx, ny, dx, dy = 30, 24, 5.0, 4.0
    dem = W.spectral_dem(nx, ny, dx, 2.2, 30.0, seed=5)
    t, Q, phi = [0.0, 100.0], [2.0, 6.0], [0.7, 0.5]
    i0, i1 = 5, 12
    for side in range(4):
        s = _sim(dem, dx, dy, W.default_params(), L)
        s.set_inflow(side, i0, i1, t, Q, phi)
        q = None
        for tt in (10.0, 60.0):
            q = np.interp(tt, t, Q) / ((i1 - i0) * (dy if side < 2 else dx))
            for k in (0, 1):  # the two ghost layers
                a = i0 + 3
                gi, gj = {0: (-1 - k, a), 1: (nx + k, a), 2: (a, -1 - k), 3: (a, ny + k)}[side]
                u = s.inflow_state(0, gi, gj, tt)
                gm = s.cell_geom(gi, gj)
                Jh = u[0] + u[3]
                assert abs(u[0] / Jh - np.interp(tt, t, phi)) < 1e-14, f"inflow solid fraction (side {side})"
                n_c, t_c = (1, 2) if side < 2 else (2, 1)
                vn = (u[n_c] + u[n_c + 3]) / Jh * (1.0 if side in (0, 2) else -1.0)
                assert vn > 0.0, f"inflow ghost moves out of the domain (side {side})"
                assert abs(Jh * vn - q) < 1e-12 * q, f"inflow ghost does not carry Q/W (side {side})"
                assert u[t_c] == 0.0 and u[t_c + 3] == 0.0, f"tangential inflow momentum (side {side})"
                cel = math.sqrt(G * gm["c"] * (gm["A11"] if side < 2 else gm["A22"]) * Jh / gm["J"])
                assert abs(vn - cel) < 1e-12 * cel, f"inflow ghost not at critical depth (side {side})"
        # outside the hydrograph's time span there is no inflow, even where its last discharge is not 0
        assert np.all(s.inflow_state(0, *{0: (-1, 8), 1: (nx, 8), 2: (8, -1), 3: (8, ny)}[side], 150.0) == 0.0)
        s.step(30)  # the other sides closed: the volume is what came in
        b = s.budget()
        for ph in ("s", "f"):
            vol = b[f"vol_{ph}"]
            assert vol > 0.0
            assert abs(vol - b[f"bnd_in_{ph}"] - b[f"clamp_{ph}"]) < 1e-12 * vol, \
                f"volume budget does not close (inflow on side {side})"


def pin_stage_times(L=None):
    """The stages sample the boundary data at their own times, as the schemes
    define them (Sect. 2.2): the two-step modified Euler at t and t + dt, the
    three-stage SSP Runge-Kutta at t, t + dt and t + dt/2.  A hydrograph that
    is non-zero only in a short window delivers mass within one step exactly
    when a stage time falls inside the window."""
    nx, ny = 20, 12
    dem = W.flat_dem(nx, ny)
    t0, dt = 10.0, 1.0

    def volume_after(rk, centre):
        p = W.default_params(rk=rk, bc=(0, 1, 0, 0))
        s = _sim(dem, 5.0, 5.0, p, L)
        w = 0.1 * dt
        s.set_inflow(0, 4, 8, [0.0, centre - 2 * w, centre - w, centre + w, centre + 2 * w, 100.0],
                     [0.0, 0.0, 3.0, 3.0, 0.0, 0.0], [0.6] * 6)
        s.t = t0
        s.step_dt(dt)
        b = s.budget()
        return b["vol_s"] + b["vol_f"]

    for rk, inside, outside in ((2, (0.0, 1.0), (0.5, 0.25)), (3, (0.0, 1.0, 0.5), (0.25, 0.75))):
        for f in inside:
            assert volume_after(rk, t0 + f * dt) > 0.0, f"rk {rk}: no stage at t + {f} dt"
        for f in outside:
            assert volume_after(rk, t0 + f * dt) == 0.0, f"rk {rk}: a stage at t + {f} dt"


def pin_time_step_cap(L=None):
    """The time step is CFL min(dx, dy) / a_max, capped at dt_max; a domain
    without motion or mass takes dt_max (Sect. 2.2).  A pure-fluid lake at
    rest on a flat bed has a_max = sqrt(g h)."""
    nx, ny, dx, dy, h = 12, 9, 5.0, 4.0, 0.5
    for dt_max in (0.05, 1.0):
        p = _pure_fluid(dt_max=dt_max, cfl=0.1)
        s = _sim(W.flat_dem(nx, ny), dx, dy, p, L)
        assert s.cfl_dt() == dt_max, "a dry domain does not take dt_max"
        s.set_release(np.full((ny, nx), h), np.zeros((ny, nx)))
        want = min(dt_max, 0.1 * min(dx, dy) / math.sqrt(G * h))
        assert abs(s.cfl_dt() - want) < 1e-14 * want, f"time step {s.cfl_dt()} != {want}"


def pin_positivity_clamp(L=None):
    """A step far beyond the CFL limit drives a cell's depth below zero: the
    depths stay >= 0 (R5), the added volume is counted, and the closed box's
    volume budget closes with it: volume(t) - volume(0) = clamp volume > 0."""
    nx, ny = 16, 12
    for rk in (2, 3):  # the RK3 step weighs its stages' clamp volumes 1/6, 1/6, 2/3
        p = _pure_fluid(bc=(0, 0, 0, 0), rk=rk)
        s = _sim(W.flat_dem(nx, ny), 5.0, 5.0, p, L)
        h = np.zeros((ny, nx))
        h[6, 7] = 0.8
        vx = np.zeros((ny, nx))
        vx[6, 7] = 2.0
        s.set_release(h, np.zeros((ny, nx)), vx_f=vx)
        v0 = s.budget()["vol_f"]
        a = 2.0 + math.sqrt(G * 0.8)
        s.step_dt(2.0 * 5.0 / a)  # the cell's outflow is twice its volume
        U = s.get_U()
        assert U[0].min() >= 0.0 and U[3].min() >= 0.0, "negative depth left by the step"
        b = s.budget()
        assert b["clamp_f"] > 0.0 and b["clamp_cells"] >= 1, "no clamp counted"
        assert abs(b["vol_f"] - v0 - b["clamp_f"]) < 1e-12 * v0, f"rk {rk}: volume budget does not close with the clamp"
    # the solid phase too, on cells with dx != dy (a clamped volume is a depth times dx dy)
    p = _pure_solid(bc=(0, 0, 0, 0), delta_b_deg=0.0)
    s = _sim(W.flat_dem(nx, ny), 5.0, 4.0, p, L)
    h = np.zeros((ny, nx))
    h[6, 7] = 0.8
    vx = np.zeros((ny, nx))
    vx[6, 7] = 2.0
    s.set_release(h, np.ones((ny, nx)), vx_s=vx)
    v0 = s.budget()["vol_s"]
    s.step_dt(2.0 * 5.0 / (2.0 + math.sqrt(G * 0.8)))
    b = s.budget()
    assert s.get_U()[0].min() >= 0.0 and b["clamp_s"] > 0.0, "no solid clamp"
    assert abs(b["vol_s"] - v0 - b["clamp_s"]) < 1e-12 * v0, "solid volume budget does not close with the clamp"


def pin_rotation_transmissive(L=None, steps=30):
    """pin_rotation with every side transmissive and water reaching every
    side from the first step: rotating the problem by 90 degrees commutes with
    the step, so the zero-gradient ghosts (R4) are the same on all four
    sides."""
    n = 32
    rng = np.random.default_rng(8)
    dem = W.spectral_dem(n, n, 5.0, 2.2, 20.0, seed=8) + rng.random((n, n))
    p = W.default_params(bc=(1, 1, 1, 1), cfl=0.2)
    h = 0.2 + 0.3 * rng.random((n, n))
    phi = rng.uniform(0.4, 0.7, (n, n))
    a = _sim(dem, 5.0, 5.0, p, L)
    a.set_release(h, phi)
    b = _sim(_rot(dem), 5.0, 5.0, p, L)
    b.set_release(_rot(h), _rot(phi))
    for _ in range(steps):
        dt = a.cfl_dt()
        a.step_dt(dt)
        b.step_dt(dt)
    Ua, Ub = a.get_U(), b.get_U()
    exp = np.stack([_rot(Ua[0]), -_rot(Ua[2]), _rot(Ua[1]), _rot(Ua[3]), -_rot(Ua[5]), _rot(Ua[4])])
    err = np.abs(Ub - exp).max() / np.abs(Ua).max()
    assert err < 1e-12, f"rotation invariance with transmissive sides broken: {err}"


def pin_rotation_rectangular(L=None, steps=30):
    """Rotation by 90 degrees with cells of different width and height: the
    rotated problem has the cell sides exchanged (dx' = dy, dy' = dx), and the
    step commutes with the rotation, so every difference along X and along Y
    (slopes, curvature, fluxes, pressure gradient) uses its own spacing."""
    n, dx, dy = 30, 5.0, 3.5
    rng = np.random.default_rng(12)
    dem = W.spectral_dem(n, n, dx, 2.2, 25.0, seed=12) + rng.random((n, n))
    p = W.default_params(bc=(1, 1, 1, 1), cfl=0.2, c_d=0.05)
    h = 0.2 + 0.3 * rng.random((n, n))
    phi = rng.uniform(0.4, 0.7, (n, n))
    a = _sim(dem, dx, dy, p, L)
    a.set_release(h, phi)
    b = _sim(_rot(dem), dy, dx, p, L)
    b.set_release(_rot(h), _rot(phi))
    for _ in range(steps):
        dt = a.cfl_dt()
        assert abs(dt - b.cfl_dt()) <= 1e-14 * dt, "rotated run takes a different dt"
        a.step_dt(dt)
        b.step_dt(dt)
    Ua, Ub = a.get_U(), b.get_U()
    exp = np.stack([_rot(Ua[0]), -_rot(Ua[2]), _rot(Ua[1]), _rot(Ua[3]), -_rot(Ua[5]), _rot(Ua[4])])
    err = np.abs(Ub - exp).max() / np.abs(Ua).max()
    assert err < 1e-12, f"rotation invariance with rectangular cells broken: {err}"


def pin_rotation_viscous(L=None, steps=20):
    """pin_rotation_rectangular with the viscous fluid term (Eq.
    SrcF_vis_Topo) on a rough bed, where A is not the identity: the face
    brackets of the X and Y derivatives must map onto each other under the
    rotation, with their own spacings and metric entries."""
    n, dx, dy = 26, 5.0, 3.5
    rng = np.random.default_rng(21)
    dem = W.spectral_dem(n, n, dx, 2.2, 25.0, seed=21) + 2.0 * rng.random((n, n))
    p = W.default_params(bc=(1, 1, 1, 1), cfl=0.2, nu_f=2.0)
    h = 0.3 + 0.3 * rng.random((n, n))
    phi = rng.uniform(0.2, 0.5, (n, n))
    vx, vy = rng.normal(0, 0.5, (n, n)), rng.normal(0, 0.5, (n, n))
    a = _sim(dem, dx, dy, p, L)
    a.set_release(h, phi, vx, vy, vy, vx)
    b = _sim(_rot(dem), dy, dx, p, L)
    # velocities rotate as (vX, vY) -> (-vY, vX)
    b.set_release(_rot(h), _rot(phi), -_rot(vy), _rot(vx), -_rot(vx), _rot(vy))
    for _ in range(steps):
        dt = a.cfl_dt()
        a.step_dt(dt)
        b.step_dt(dt)
    Ua, Ub = a.get_U(), b.get_U()
    exp = np.stack([_rot(Ua[0]), -_rot(Ua[2]), _rot(Ua[1]), _rot(Ua[3]), -_rot(Ua[5]), _rot(Ua[4])])
    err = np.abs(Ub - exp).max() / np.abs(Ua).max()
    assert err < 1e-12, f"rotation invariance with the viscous term broken: {err}"


def pin_max_speed_everywhere(L=None):
    """a_max is the largest local speed over every cell (R7), including the
    last column and the last row; a solid layer without fluid moving at v on a
    flat bed has the speed v + sqrt(g (1 - alpha) h) (the solid celerity
    carries the buoyancy factor 1 - rho_f / rho_s)."""
    nx, ny = 9, 7
    for (j, i) in ((3, nx - 1), (ny - 1, 4), (ny - 1, nx - 1)):
        h = np.full((ny, nx), 0.5)
        h[j, i] = 2.0
        s = _sim(W.flat_dem(nx, ny), 5.0, 4.0, _pure_fluid(), L)
        s.set_release(h, np.zeros((ny, nx)))
        assert abs(s.max_speed() - math.sqrt(G * 2.0)) < 1e-14, f"a_max misses cell ({i}, {j})"
    p = W.default_params()  # rho_f / rho_s = 1100 / 2700
    al = p["rho_f"] / p["rho_s"]
    one = np.ones((ny, nx))
    s = _sim(W.flat_dem(nx, ny), 5.0, 5.0, p, L)
    s.set_release(1.5 * one, one, 12.0 * one, 0 * one)
    want = 12.0 + math.sqrt(G * (1.0 - al) * 1.5)
    assert abs(s.max_speed() - want) < 1e-13 * want, f"solid speed {s.max_speed()} != {want}"


def pin_max_speed_rows(L=None):
    """The largest wave speed over a range of rows [j0, j1) (the strip of a
    row-decomposed domain takes the CFL maximum of its own rows, Sect. 2.2):
    with one fast cell in row r of a still fluid layer on a flat bed (speed
    sqrt(g h)), a range holds the fast speed exactly when it holds row r,
    the first and the last row included, and every range's maximum is the
    largest of its rows' own."""
    nx, ny = 7, 9
    slow, fast = math.sqrt(G * 0.5), math.sqrt(G * 2.0)
    for r in (0, 4, ny - 1):
        h = np.full((ny, nx), 0.5)
        h[r, 3] = 2.0
        s = _sim(W.flat_dem(nx, ny), 5.0, 4.0, _pure_fluid(), L)
        s.set_release(h, np.zeros((ny, nx)))
        for j0 in range(ny):
            for j1 in range(j0 + 1, ny + 1):
                want = fast if j0 <= r < j1 else slow
                got = s.max_speed_rows(j0, j1)
                assert abs(got - want) < 1e-14 * want, f"rows [{j0}, {j1}) with the fast row {r}: {got} != {want}"
        assert abs(s.max_speed_rows(0, ny) - s.max_speed()) < 1e-15 * fast


def pin_step_amax(L=None):
    """A step whose CFL time step comes from a given largest speed (a strip of
    a decomposed domain steps with the whole domain's a_max, Sect. 2.2): with
    the simulation's own a_max it is the ordinary step, bit for bit; with
    another speed a its time step is CFL min(dx, dy) / a, and the state is the
    step with that prescribed time step."""
    nx, ny = 24, 16
    cfg = W.release_config(nx=nx, ny=ny, dx=5.0)
    dx, dy = 5.0, 4.0
    cfl = cfg["params"]["cfl"]
    def fresh():
        s = _sim(cfg["dem"], dx, dy, cfg["params"], L)
        s.set_release(cfg["h"], cfg["phi_s"])
        s.step(3)
        return s
    a, b = fresh(), fresh()
    amax = a.max_speed()
    dt_a = a.step_amax(amax)
    b.step(1)
    assert np.array_equal(a.get_U(), b.get_U()) and dt_a == b.last_dt, "step_amax with the own a_max is not the step"
    for scale in (2.0, 3.5):
        c, d = fresh(), fresh()
        speed = scale * c.max_speed()
        dt_c = c.step_amax(speed)
        want = cfl * min(dx, dy) / speed
        assert abs(dt_c - want) < 1e-15 * want, f"dt {dt_c} != CFL min(dx, dy) / a = {want}"
        d.step_dt(dt_c)
        assert np.array_equal(c.get_U(), d.get_U()), "step_amax is not the step with its own time step"


def pin_step_composition(L=None):
    """The two-step modified Euler (Sect. 2.2) and the three-stage SSP
    Runge-Kutta are convex combinations of single stages S (U + dt L(U) with
    friction, clamp and the dry rule), with the dry rule (R5) applied to every
    combined state:
    - Heun: U' = D((U + S(S(U, t), t + dt)) / 2);
    - RK3: W = D(3/4 U + 1/4 S(S(U, t), t + dt)), then U' = D(U/3 + 2/3 S(W, t + dt/2)).
    Here D zeroes a phase's momentum where its mass is <= J h_dry.  The
    oracle's whole step is checked against this composition of its
    single-stage call.  The state is thin films near h_dry, where the dry rule
    of the combinations decides."""
    nx, ny, dt, t0 = 24, 18, 0.05, 3.0
    rng = np.random.default_rng(31)
    dem = W.spectral_dem(nx, ny, 2.0, 2.2, 3.0, seed=31) + 0.2 * rng.random((ny, nx))
    for rk in (2, 3):
        p = W.default_params(rk=rk, bc=(0, 1, 1, 0), h_dry=0.01)
        s = _sim(dem, 2.0, 2.0, p, L)
        J = s.geometry()["J"]
        U = np.zeros((6, ny, nx))
        for ph in (0, 1):
            m = J * p["h_dry"] * rng.uniform(0.0, 3.0, (ny, nx)) * (rng.random((ny, nx)) < 0.7)
            U[3 * ph] = m
            wet = m > J * p["h_dry"]
            U[3 * ph + 1] = np.where(wet, m * rng.normal(0, 1.0, (ny, nx)), 0.0)
            U[3 * ph + 2] = np.where(wet, m * rng.normal(0, 1.0, (ny, nx)), 0.0)

        def D(V):
            V = V.copy()
            for ph in (0, 1):
                dry = V[3 * ph] <= J * p["h_dry"]
                V[3 * ph + 1][dry] = 0.0
                V[3 * ph + 2][dry] = 0.0
            return V

        def S(V, tt):
            s.set_U(V)
            return s.stage(tt, dt)

        if rk == 2:
            want = D(0.5 * (U + S(S(U, t0), t0 + dt)))
        else:
            Wc = D(0.75 * U + 0.25 * S(S(U, t0), t0 + dt))
            want = D(U / 3.0 + 2.0 * S(Wc, t0 + 0.5 * dt) / 3.0)
        s.set_U(U)
        s.t = t0
        s.step_dt(dt)
        got = s.get_U()
        err = np.abs(got - want).max() / np.abs(want).max()
        assert err < 1e-13, f"rk {rk}: the step is not the composition of its stages ({err})"


def pin_phase_symmetry(L=None, steps=20):
    """With rho_f = 0 (alpha = 0) and delta_b = 0 the solid's equations are
    the fluid's (App. A): the same pressure, celerity and basal pressure with
    its centripetal term, no buoyancy, friction or drag, and no fluid basal
    friction (k_f = 0).  So a pure solid and a pure fluid with the same depth
    and velocity evolve identically, component for component, on a rough bed
    fast enough that the layer lifts off in places (p_b clamped at 0)."""
    n = 28
    rng = np.random.default_rng(17)
    c = (np.arange(n) + 0.5) * 1.0
    X, Y = np.meshgrid(c, c)
    # bumps of curvature ~0.6 / m: at 8 m/s, v^2 kappa > g c on the crests
    dem = 0.5 * np.sin(2 * np.pi * X / 8.0) * np.sin(2 * np.pi * Y / 8.0) + 0.05 * rng.random((n, n))
    p = W.default_params(rho_f=0.0, delta_b_deg=0.0, k_f=0.0, bc=(0, 1, 1, 0), cfl=0.2)
    h = 0.3 + 0.4 * rng.random((n, n))
    vx, vy = 8.0 + rng.normal(0, 1.0, (n, n)), rng.normal(0, 2.0, (n, n))
    zero = np.zeros((n, n))
    a = _sim(dem, 1.0, 1.0, p, L)
    a.set_release(h, np.ones((n, n)), vx, vy, zero, zero)
    b = _sim(dem, 1.0, 1.0, p, L)
    b.set_release(h, zero, zero, zero, vx, vy)
    for _ in range(steps):
        dt = a.cfl_dt()
        assert abs(dt - b.cfl_dt()) <= 1e-14 * dt, "the two phases take different time steps"
        a.step_dt(dt)
        b.step_dt(dt)
    Ua, Ub = a.get_U(), b.get_U()
    err = np.abs(Ua[0:3] - Ub[3:6]).max() / np.abs(Ua).max()
    assert err < 1e-12, f"solid and fluid phases differ: {err}"
    assert np.abs(Ua[3:6]).max() == 0.0 and np.abs(Ub[0:3]).max() == 0.0


def pin_inflow_mirror(L=None, steps=60):
    """Mirror symmetry with inflow (Sect. 3.1.2, Mode II): an inflow on the
    west side of a terrain and the same inflow on the east side of the
    terrain mirrored in X give mirrored states, with the X momenta negated.
    The same holds for south and north in Y.  Both ghost layers of every side
    then carry the inflow state alike."""
    nx, ny = 36, 28
    rng = np.random.default_rng(19)
    dem = W.spectral_dem(nx, ny, 4.0, 2.2, 12.0, seed=19) + rng.random((ny, nx))
    p = W.default_params(bc=(0, 0, 0, 0), cfl=0.2)
    t, Q, phi = [0.0, 30.0, 200.0], [4.0, 9.0, 0.0], [0.6, 0.5, 0.5]
    for axis, (sa, sb), (i0, i1) in ((1, (0, 1), (9, 17)), (0, (2, 3), (12, 22))):
        da = dem
        db = dem[:, ::-1].copy() if axis == 1 else dem[::-1, :].copy()
        a = _sim(da, 4.0, 4.0, p, L)
        a.set_inflow(sa, i0, i1, t, Q, phi)
        b = _sim(db, 4.0, 4.0, p, L)
        b.set_inflow(sb, i0, i1, t, Q, phi)
        for _ in range(steps):
            dt = a.cfl_dt()
            assert abs(dt - b.cfl_dt()) <= 1e-14 * dt, "mirrored run takes a different dt"
            a.step_dt(dt)
            b.step_dt(dt)
        Ua, Ub = a.get_U(), b.get_U()
        flip = (lambda f: f[:, ::-1]) if axis == 1 else (lambda f: f[::-1, :])
        neg = (1, 4) if axis == 1 else (2, 5)
        exp = np.stack([-flip(Ua[c]) if c in neg else flip(Ua[c]) for c in range(6)])
        assert np.abs(Ua[0]).max() > 0.0
        err = np.abs(Ub - exp).max() / np.abs(Ua).max()
        assert err < 1e-12, f"inflow mirror symmetry broken (sides {sa}, {sb}): {err}"


def pin_uniform_flow_viscous(L=None):
    """A uniform mixture flow (both phases at one velocity, no basal
    friction) on a flat bed with transmissive sides has no gradient anywhere,
    corners included.  One stage with the viscous term on leaves every cell
    unchanged: the fluxes are uniform, the basal normal has no horizontal
    part, the drag vanishes and the viscous brackets vanish."""
    nx, ny = 14, 11
    one = np.ones((ny, nx))
    p = W.default_params(bc=(1, 1, 1, 1), nu_f=1.5, delta_b_deg=0.0)  # no basal friction
    s = _sim(W.flat_dem(nx, ny), 2.0, 3.0, p, L)
    s.set_release(0.8 * one, 0.4 * one, 1.2 * one, -0.7 * one, 1.2 * one, -0.7 * one)
    U0 = s.get_U()
    out = s.stage(0.0, 0.05)
    err = np.abs(out - U0).max() / np.abs(U0).max()
    assert err < 1e-14, f"a uniform flow changed: {err}"


def pin_thin_film_has_no_velocity(L=None):
    """The dry rule (R5) is a threshold on the normal thickness h = U / J,
    not on U: a phase thinner than h_dry carries no velocity, on a 45 degree
    plane (J = sqrt 2) as on a flat bed.  A film thinner than h_dry
    everywhere, with momenta set on it, moves its mass in one stage exactly
    as the same film without momenta: every face state is thinner than
    h_dry, so no face has a velocity."""
    nx, ny = 16, 12
    rng = np.random.default_rng(27)
    p = W.default_params(bc=(1, 1, 1, 1), h_dry=0.01)
    dem = W.incline_dem(nx, ny, 1.0, 1.0, 45.0)
    # thinner than h_dry, but J h above h_dry: a threshold on U would give it a velocity
    h = p["h_dry"] * rng.uniform(0.75, 0.98, (ny, nx))
    for phi_s in (0.0, 1.0):  # a pure fluid and a pure solid film
        outs = []
        for v in (0.0, 1.0):
            s = _sim(dem, 1.0, 1.0, p, L)
            s.set_release(h, np.full((ny, nx), phi_s), v * rng.normal(0, 2.0, (ny, nx)),
                          v * rng.normal(0, 2.0, (ny, nx)), v * rng.normal(0, 2.0, (ny, nx)),
                          v * rng.normal(0, 2.0, (ny, nx)))
            outs.append(s.stage(0.0, 0.01))
        for c in (0, 3):
            assert np.array_equal(outs[0][c], outs[1][c]), "momenta of a film thinner than h_dry moved mass"


def pin_clamp_count(L=None):
    """The clamp-cell count of a Heun step is the number of phase masses set
    to 0 by the positivity clamp in each of its two stages.  A stage never
    drives a massless cell negative: the central flux moves mass into a dry
    cell, not out of it.  So a mass that is positive before a stage and
    exactly 0 after it was clamped.  The two stages are taken one by one
    through the single-stage call and their clamps counted, and the step's
    count must be their sum."""
    nx, ny = 16, 12
    s = _sim(W.flat_dem(nx, ny), 5.0, 5.0, _pure_fluid(bc=(0, 0, 0, 0)), L)
    h = np.zeros((ny, nx))
    h[6, 7], h[3, 3] = 0.8, 0.5
    vx = np.zeros((ny, nx))
    vx[6, 7], vx[3, 3] = 2.0, -1.0
    s.set_release(h, np.zeros((ny, nx)), vx_f=vx)
    U = s.get_U()
    dt = 2.0 * 5.0 / (2.0 + math.sqrt(G * 0.8))

    def clamped(before, after):
        return sum(int(np.count_nonzero((before[c] > 0.0) & (after[c] == 0.0))) for c in (0, 3))

    W1 = s.stage(0.0, dt)
    s.set_U(W1)
    W2 = s.stage(dt, dt)
    want = clamped(U, W1) + clamped(W1, W2)
    assert clamped(U, W1) >= 1
    s.set_U(U)
    s.step_dt(dt)
    assert s.budget()["clamp_cells"] == want, f"clamp count {s.budget()['clamp_cells']} != {want}"


def pin_viscous_only_where_the_fluid_is_wet(L=None):
    """The viscous term (Eq. SrcF_vis_Topo) is a force on the fluid phase
    where it moves; a cell whose fluid is thinner than h_dry has no fluid
    velocity (R5) and gets no viscous force, even where a neighbour's sheared
    fluid gives it velocity gradients and its fluid becomes wet within the
    stage.  One stage with and without viscosity gives the same fluid
    momenta on every cell whose fluid was thin."""
    n = 24
    p0 = W.default_params(bc=(1, 1, 1, 1), h_dry=0.01, delta_b_deg=0.0)
    c = (np.arange(n) + 0.5) * 1.0
    X, Y = np.meshgrid(c, c)
    wet = X < n / 2
    hs = np.full((n, n), 0.5)
    hf = np.where(wet, 0.3, 0.5 * p0["h_dry"])
    h = hs + hf
    phi = hs / h
    vyf = np.where(wet, 1.5 * np.sin(2 * np.pi * X / 8.0), 0.0)
    zero = np.zeros((n, n))
    outs = []
    for nu in (0.0, 2.0):
        s = _sim(W.flat_dem(n, n), 1.0, 1.0, dict(p0, nu_f=nu), L)
        s.set_release(h, phi, zero, zero, zero, vyf)
        outs.append(s.stage(0.0, 0.02))
    thin = ~wet
    assert np.any(outs[0][3][thin] > s.geometry()["J"][thin] * p0["h_dry"]), "no thin cell became wet"
    for comp in (4, 5):
        assert np.array_equal(outs[0][comp][thin], outs[1][comp][thin]), "viscous force on a cell without fluid velocity"
    assert not np.array_equal(outs[0][5][wet], outs[1][5][wet])


def pin_thin_cell_has_no_phase_fractions(L=None):
    """A cell thinner than h_dry in total has no phase fractions (R5), so no
    pressure-gradient source acts on it, whichever fraction the fluid's source
    carries (phi^s by reading R1, or phi^f as printed in Eq. SrcF_f_Topo).
    Next to a deep mixture, where grad P is large and the thin cells become
    wet within the stage, one stage in the two forms gives the same fluid
    momenta on every cell that was thin."""
    n = 20
    p0 = W.default_params(bc=(1, 1, 1, 1), h_dry=0.01, delta_b_deg=0.0)
    c = (np.arange(n) + 0.5) * 1.0
    X, _ = np.meshgrid(c, c)
    deep = X < n / 2
    h = np.where(deep, 1.0 + 0.05 * X, 0.6 * p0["h_dry"])
    phi = np.full((n, n), 0.6)
    outs = []
    for mode in (0, 1):
        s = _sim(W.flat_dem(n, n), 1.0, 1.0, dict(p0, fluid_pg_mode=mode), L)
        s.set_release(h, phi)
        outs.append(s.stage(0.0, 0.02))
    thin = ~deep
    J = s.geometry()["J"]
    assert np.any(outs[0][3][thin] > J[thin] * p0["h_dry"]), "no thin cell became wet"
    for comp in (4, 5):
        assert np.array_equal(outs[0][comp][thin], outs[1][comp][thin]), "pressure-gradient source on a thin cell"
    assert not np.array_equal(outs[0][4][deep], outs[1][4][deep])


def pin_budget_sums(L=None):
    """The budgets' volumes and momenta are the sums of the six conserved
    fields times the cell area (a10: sum U dx dy per component), each field
    to its own entry, after a few steps of a flow on rectangular cells."""
    nx, ny, dx, dy = 21, 17, 4.0, 3.0
    rng = np.random.default_rng(41)
    dem = W.spectral_dem(nx, ny, dx, 2.2, 10.0, seed=41)
    s = _sim(dem, dx, dy, W.default_params(bc=(0, 1, 1, 0)), L)
    s.set_release(0.3 + rng.random((ny, nx)), rng.uniform(0.3, 0.7, (ny, nx)), rng.normal(0, 1, (ny, nx)),
                  rng.normal(0, 1, (ny, nx)), rng.normal(0, 1, (ny, nx)), rng.normal(0, 1, (ny, nx)))
    s.step(5)
    U, b = s.get_U(), s.budget()
    for key, c in (("vol_s", 0), ("mom_xs", 1), ("mom_ys", 2), ("vol_f", 3), ("mom_xf", 4), ("mom_yf", 5)):
        want = math.fsum(U[c].ravel()) * dx * dy
        assert abs(b[key] - want) <= 1e-12 * max(abs(want), math.fsum(np.abs(U[c]).ravel()) * dx * dy), \
            f"budget {key} is not the sum of field {c}"


def pin_step_clock(L=None):
    """A CFL step takes dt = CFL min(dx, dy) / a_max of the state it starts
    from (Sect. 2.2): for a pure-fluid lake at rest on a flat bed that is CFL
    min(dx, dy) / sqrt(g h).  The clock advances by the steps' dts and the
    step count by one per step, for both time integrators."""
    nx, ny, dx, dy, h = 10, 8, 5.0, 4.0, 0.5
    for rk in (2, 3):
        s = _sim(W.flat_dem(nx, ny), dx, dy, _pure_fluid(cfl=0.1, rk=rk), L)
        s.set_release(np.full((ny, nx), h), np.zeros((ny, nx)))
        dts = s.step(1)
        want = 0.1 * min(dx, dy) / math.sqrt(G * h)
        assert abs(dts[0] - want) < 1e-14 * want and abs(s.last_dt - want) < 1e-14 * want, \
            f"rk {rk}: the step's dt {dts[0]} != {want}"
        dts = np.concatenate([dts, s.step(6)])
        b = s.budget()
        assert b["steps"] == 7, f"rk {rk}: step count {b['steps']}"
        assert abs(b["t"] - math.fsum(dts)) < 1e-14 * b["t"], f"rk {rk}: clock {b['t']} != sum of dts"

# ----------------------------------------------------------------------------
# Coulomb friction and the curvature term in the basal pressure


def _slide_on_plane(p, buoy, L):
    """One stage of a uniform solid layer sliding on a 30 deg plane (delta_b =
    20 deg) up and down the slope: the X momentum changes by
    dt h g buoy (sin z -+ cos z tan d)."""
    zeta, delta, h, dt = 30.0, 20.0, 2.0, 0.05
    tz, td = math.radians(zeta), math.radians(delta)
    nx, ny, dx = 8, 6, 2.0
    one = np.ones((ny, nx))
    for vs in (4.0, -4.0):
        s = _sim(W.incline_dem(nx, ny, dx, dx, zeta), dx, dx, p, L)
        s.set_release(h * one, one, vs * math.cos(tz) * one, 0 * one)
        U0 = s.get_U()
        out = s.stage(0.0, dt)
        dq = buoy * G * h * (math.sin(tz) - math.copysign(1.0, vs) * math.cos(tz) * math.tan(td))
        assert np.allclose(out[1], U0[1] + dt * dq, rtol=1e-12, atol=0), "slide on a plane: wrong acceleration"
        assert np.abs(out[2]).max() == 0.0


def pin_friction_buoyant(L=None):
    """The slide of pin_friction with the default densities: the solid's
    basal pressure carries the buoyancy factor 1 - alpha (alpha = rho_f /
    rho_s, Eq. Src_nd_Topo), which scales the drive and the friction alike."""
    p = W.default_params(delta_b_deg=20.0, bc=(W.BC_TRANSMISSIVE,) * 4)
    _slide_on_plane(p, 1.0 - p["rho_f"] / p["rho_s"], L)


def pin_friction(L=None):
    """(a) A uniform pure-solid layer sliding on a 30 deg plane (delta_b = 20
    deg): one stage changes J h^s v_X^s = h v_s by dt h g (sin z -+ cos z tan d)
    (friction opposes the motion, downslope or upslope).  (b) At the bottom of
    a concave parabolic bed of radius R the basal pressure is h (g + V^2/R)
    (centripetal term, Eq. Src_nd_Topo with kappa < 0), so one stage removes
    dt h (g + V^2/R) tan d of momentum.  (c) Over a convex crest with V^2/R > g
    the layer lifts off: p_b is clamped at 0 and no friction acts."""
    delta, h, dt, dx = 20.0, 2.0, 0.05, 2.0
    td = math.radians(delta)
    p = _pure_solid(delta_b_deg=delta, bc=(W.BC_TRANSMISSIVE,) * 4)
    _slide_on_plane(p, 1.0, L)
    R, V = 10.0, 12.0
    nx = 21
    x = (np.arange(nx) + 0.5) * dx
    X0 = x[nx // 2]
    for sign in (1.0, -1.0):
        dem = np.broadcast_to(sign * (x - X0) ** 2 / (2 * R), (3, nx)).copy()
        q = _sim(dem, dx, dx, p, L)
        U = np.zeros((6, 3, nx))
        U[0] = h
        U[1] = h * V
        q.set_U(U)
        out = q.stage(0.0, dt)
        got = out[1, 1, nx // 2]
        if sign > 0:
            exp = h * V - dt * h * (G + V * V / R) * math.tan(td)
            assert abs(got - exp) < 1e-12 * h * V, f"centripetal basal pressure: {got} vs {exp}"
        else:
            assert V * V / R > G
            assert abs(got - h * V) < 1e-12 * h * V, "lift-off: friction must vanish when p_b < 0"


def pin_closed_box(L=None, steps=400):
    """A mixture column released in the middle of a closed box on an oblique
    plane reaches all four walls; each phase's volume is conserved to
    round-off and the clamp never fires at CFL 0.1."""
    nx, ny, dx = 30, 24, 2.0
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dx
    X, Y = np.meshgrid(x, y)
    dem = 0.04 * X + 0.03 * Y
    h = W.parabolic_cap(nx, ny, dx, dx, 15, 12, 6, 4.0)
    s = _sim(dem, dx, dx, W.default_params(cfl=0.1, delta_b_deg=10.0), L)
    s.set_release(h, np.full((ny, nx), 0.55))
    b0 = s.budget()
    s.step(steps)
    b = s.budget()
    pr = s.primitive()
    assert min(pr["h"][:, 0].max(), pr["h"][:, -1].max(), pr["h"][0].max(), pr["h"][-1].max()) > 1e-3, \
        "flow did not reach every wall"
    assert b["clamp_cells"] == 0
    for ph in ("s", "f"):
        rel = abs(b[f"vol_{ph}"] - b0[f"vol_{ph}"]) / b0[f"vol_{ph}"]
        assert rel < 1e-13, f"closed box: phase {ph} volume drift {rel}"


# ----------------------------------------------------------------------------
# fluid viscosity (Eq. SrcF_vis_Topo) and fluid basal friction (Eq. SrcF_nd_Topo)


def pin_viscous(L=None):
    """On a flat bed (A = I, J = 1) with uniform depth the viscous source of a
    sinusoidal shear or stretch of the fluid velocity is nu phi^f times
    h v'' (shear) or 2 h v'' (stretch along the component's own axis), with
    v'' = -k^2 v; second-order accurate at 32 cells per wavelength."""
    n, dx, h, V, nu, dt = 64, 1.0, 1.5, 0.8, 0.3, 1e-3
    k = 2 * math.pi / (32 * dx)
    c = (np.arange(n) + 0.5) * dx
    Xc, Yc = np.meshgrid(c, c)
    cases = (("vx_f", Yc, 4, 1.0), ("vx_f", Xc, 4, 2.0), ("vy_f", Xc, 5, 1.0), ("vy_f", Yc, 5, 2.0))
    for name, coord, comp, factor in cases:
        outs = []
        for nuv in (0.0, nu):
            p = _pure_fluid(nu_f=nuv, bc=(W.BC_TRANSMISSIVE,) * 4)
            s = _sim(W.flat_dem(n, n), dx, dx, p, L)
            vel = {"vx_f": None, "vy_f": None}
            vel[name] = V * np.sin(k * coord)
            s.set_release(np.full((n, n), h), np.zeros((n, n)), None, None, vel["vx_f"], vel["vy_f"])
            outs.append(s.stage(0.0, dt)[comp])
        S = (outs[1] - outs[0]) / dt
        ex = -factor * nu * h * k * k * V * np.sin(k * coord)
        inner = (slice(6, n - 6), slice(6, n - 6))
        err = np.abs(S[inner] - ex[inner]).max() / np.abs(ex[inner]).max()
        assert err < 5e-3, f"viscous term {name}({'Y' if coord is Yc else 'X'}): error {err}"


def pin_fluid_friction(L=None):
    """Uniform pure-fluid flow on a flat bed with fluid basal friction k_f:
    dv/dt = -k_f v, so v is multiplied by the Heun factor 1 - z + z^2/2,
    z = k_f dt, at each step."""
    n, kf, dt = 6, 0.5, 0.1
    one = np.ones((n, n))
    s = _sim(W.flat_dem(n, n), 5.0, 5.0, _pure_fluid(k_f=kf, bc=(W.BC_TRANSMISSIVE,) * 4), L)
    s.set_release(2.0 * one, 0 * one, None, None, 3.0 * one, -2.0 * one)
    for _ in range(10):
        s.step_dt(dt)
    z = kf * dt
    fac = (1 - z + z * z / 2) ** 10
    pr = s.primitive()
    assert np.allclose(pr["vx_f"], 3.0 * fac, rtol=1e-13) and np.allclose(pr["vy_f"], -2.0 * fac, rtol=1e-13)


def pin_mixture_no_separation(L=None):
    """A uniform mixture (phi^s = 0.6) at rest on a flat, frictionless bed with
    a linear depth gradient moves as one fluid: the solid's own pressure
    (factor 1 - alpha_rho) plus its buoyancy (alpha_rho phi^s grad P, Eq.
    Src_f_Topo) and the fluid's pressure minus the reaction phi^s grad P (R1)
    give both phases the acceleration -g dh/dX, so no drag arises."""
    nx, ny, dx, dt, slope = 40, 5, 2.0, 0.02, 0.01
    x = (np.arange(nx) + 0.5) * dx
    h = np.broadcast_to(2.0 + slope * x, (ny, nx)).copy()
    p = W.default_params(delta_b_deg=0.0, bc=(W.BC_TRANSMISSIVE,) * 4)
    s = _sim(W.flat_dem(nx, ny), dx, dx, p, L)
    s.set_release(h, np.full((ny, nx), 0.6))
    out = s.stage(0.0, dt)
    inner = (slice(None), slice(4, nx - 4))
    vs = out[1][inner] / out[0][inner]
    vf = out[4][inner] / out[3][inner]
    ex = -dt * G * slope
    assert np.allclose(vs, ex, rtol=1e-12, atol=0), f"solid acceleration {vs.flat[0] / dt} vs {ex / dt}"
    assert np.allclose(vf, ex, rtol=1e-12, atol=0), f"fluid acceleration {vf.flat[0] / dt} vs {ex / dt}"


# ----------------------------------------------------------------------------
# central-upwind flux (scheme 1): one-sided local speeds


def pin_cu_upwind_dependence(L=None):
    """Supercritical flow (all waves move one way): the central-upwind flux
    through a face is the flux of its upwind side alone, so the stage result
    of cell k does not depend on cell k + 2 downstream (it enters only the
    downstream side of face k + 1/2); the central flux does depend on it.
    Both directions of flow and both grid directions."""
    n, dx, h0, v = 24, 5.0, 0.1, 10.0  # Froude ~ 10
    k = 10
    for axis in (0, 1):
        for sgn in (1.0, -1.0):
            for scheme, must_vary in ((1, False), (0, True)):
                outs = []
                for bump in (0.0, 0.01):
                    h = h0 * (1.0 + 0.05 * np.sin(np.arange(n) * 0.7))
                    kd = k + 2 if sgn > 0 else k - 2  # the downstream neighbour's neighbour
                    h[kd] += bump
                    hh = np.tile(h, (3, 1)) if axis == 0 else np.tile(h[:, None], (1, 3))
                    ny_, nx_ = hh.shape
                    vel = np.full(hh.shape, sgn * v)
                    p = _pure_fluid(cfl=0.1, scheme=scheme, bc=(1, 1, 1, 1))
                    s = _sim(W.flat_dem(nx_, ny_), dx, dx, p, L)
                    zero = np.zeros(hh.shape)
                    if axis == 0:
                        s.set_release(hh, zero, None, None, vel, zero)
                    else:
                        s.set_release(hh, zero, None, None, zero, vel)
                    outs.append(s.stage(0.0, 0.01))
                a, b = outs
                sel = (slice(None), 1, k) if axis == 0 else (slice(None), k, 1)
                dmax = np.abs(a[sel] - b[sel]).max()
                if must_vary:
                    assert dmax > 1e-8, f"central flux unexpectedly upwind (axis {axis})"
                else:
                    assert dmax <= 1e-15 * np.abs(a[sel]).max(), f"central-upwind flux not upwind: {dmax}"


def pin_cu_conservation_and_ritter(L=None):
    """Central-upwind form: each phase's volume is conserved to round-off in a
    closed box; the Ritter dam break converges, no less accurately than the
    central flux at the same resolution (its numerical diffusion is smaller)."""
    cfg = W.release_config(nx=48, ny=64, cfl=0.1, scheme=1)
    s = _sim(cfg["dem"], cfg["dx"], cfg["dy"], cfg["params"], L)
    s.set_release(cfg["h"], cfg["phi_s"])
    b0 = s.budget()
    s.step(150)
    b = s.budget()
    for ph in ("s", "f"):
        assert abs(b[f"vol_{ph}"] - b0[f"vol_{ph}"]) < 1e-13 * b0[f"vol_{ph}"], f"CU volume drift ({ph})"
    e10 = _ritter_error(L, 10.0, scheme=1)
    e5 = _ritter_error(L, 5.0, scheme=1)
    k5 = _ritter_error(L, 5.0, scheme=0)
    assert e5 < 0.75 * e10, f"CU Ritter error does not converge: {e10} -> {e5}"
    assert e5 <= 1.02 * k5, f"CU Ritter error {e5} above the central scheme's {k5}"


def pin_cu_rotation(L=None):
    """Rotation by 90 degrees commutes with the central-upwind step."""
    n = 32
    cfg = W.release_config(nx=n, ny=n, cfl=0.2, scheme=1)
    rng = np.random.default_rng(4)
    phi = rng.uniform(0.4, 0.7, (n, n))
    h = cfg["h"] * (1 + 0.2 * rng.random((n, n)))
    dem = cfg["dem"] + rng.random((n, n))
    a = _sim(dem, 5.0, 5.0, cfg["params"], L)
    a.set_release(h, phi)
    b = _sim(_rot(dem), 5.0, 5.0, cfg["params"], L)
    b.set_release(_rot(h), _rot(phi))
    for _ in range(30):
        dt = a.cfl_dt()
        a.step_dt(dt)
        b.step_dt(dt)
    Ua, Ub = a.get_U(), b.get_U()
    exp = np.stack([_rot(Ua[0]), -_rot(Ua[2]), _rot(Ua[1]), _rot(Ua[3]), -_rot(Ua[5]), _rot(Ua[4])])
    err = np.abs(Ub - exp).max() / np.abs(Ua).max()
    assert err < 1e-12, f"CU rotation invariance broken: {err}"


# ----------------------------------------------------------------------------
# third-order WENO reconstruction (recon 1) and three-stage SSP Runge-Kutta
# (rk 3), the options Sect. 2.2 names beside minmod and the two-step Euler


def _linear_U(nx, ny, dx):
    """Six conserved fields, each linear in X and Y (positive masses)."""
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dx
    X, Y = np.meshgrid(x, y)
    return np.stack([1.2 + 0.002 * X + 0.001 * Y, 0.5 + 0.003 * X - 0.002 * Y, -0.3 + 0.001 * X + 0.004 * Y,
                     0.9 - 0.001 * X + 0.002 * Y, 0.2 - 0.002 * X + 0.001 * Y, 0.4 + 0.001 * X - 0.003 * Y])


def pin_weno_linear_exact(L=None):
    """On data linear in X and Y both reconstructions are exact (minmod of
    two equal differences returns it; both WENO candidates are exact), so a
    stage with WENO equals the minmod stage wherever the stencil sees only
    linear data (cells two or more away from the boundary): a wrong candidate
    or face formula breaks the equality."""
    nx, ny, dx = 14, 11, 5.0
    dem = W.incline_dem(nx, ny, dx, dx, 10.0, "y")
    U = _linear_U(nx, ny, dx)
    outs = []
    for recon in (0, 1):
        s = _sim(dem, dx, dx, W.default_params(recon=recon, bc=(1, 1, 1, 1)), L)
        s.set_U(U)
        outs.append(s.stage(0.0, 0.02))
    a, b = outs
    sl = (slice(None), slice(2, ny - 2), slice(2, nx - 2))
    err = np.abs(a[sl] - b[sl]).max() / np.abs(a[sl]).max()
    assert err < 1e-13, f"WENO not exact on linear data: {err}"
    # away from linear data the two differ
    U2 = U * (1 + 0.2 * np.sin(np.arange(nx) * 1.3))[None, None, :]
    res = []
    for recon in (0, 1):
        s = _sim(dem, dx, dx, W.default_params(recon=recon, bc=(1, 1, 1, 1)), L)
        s.set_U(U2)
        res.append(s.stage(0.0, 0.02))
    assert np.abs(res[0] - res[1]).max() > 1e-8


def pin_weno_rk3_dam_break(L=None):
    """Ritter dam break with WENO and the three-stage Runge-Kutta: converges
    (error down by a quarter from 200 to 400 cells), stays below 1 % at 400
    cells, and is essentially non-oscillatory: WENO is not TVD, so the depth
    may exceed its initial maximum, but by less than 1e-5 of it and less at
    the finer grid."""
    e10, m10 = _ritter_error(L, 10.0, recon=1, rk=3, want_max=True)
    e5, m5 = _ritter_error(L, 5.0, recon=1, rk=3, want_max=True)
    assert e5 < 0.01, f"WENO/RK3 Ritter L1 error {e5} at 400 cells"
    assert e5 < 0.75 * e10, f"WENO/RK3 Ritter error does not converge: {e10} -> {e5}"
    assert m10 - 10.0 < 1e-4 and m5 - 10.0 < m10 - 10.0 + 1e-12, f"overshoot {m10 - 10.0}, {m5 - 10.0}"


def _smooth_hump(L, n, recon, rk, t_end=20.0, length=2000.0):
    dx = length / n
    x = (np.arange(n) + 0.5) * dx - length / 2
    f = lambda z: 1.0 + 0.1 * np.exp(-(z / 150.0) ** 2)
    h = (f(x - dx / 2) + 4 * f(x) + f(x + dx / 2)) / 6  # cell averages (Simpson)
    s = _sim(W.flat_dem(n, 1), dx, dx, _pure_fluid(recon=recon, rk=rk, bc=(1, 1, 1, 1)), L)
    s.set_release(h[None, :], np.zeros((1, n)))
    dt = 0.025 * dx
    for _ in range(int(round(t_end / dt))):
        s.step_dt(dt)
    return s.primitive()["h"][0]


def pin_weno_smooth_order(L=None):
    """A smooth hump of water spreading on a flat bed, self-convergence
    against the same scheme on a 4x (WENO) finer grid: halving the cells
    divides the L1 error by more than 5.5 with WENO and RK3 (third order in
    space; measured 6.8), by less than 4.5 with minmod (measured 3.8)."""
    def ratio(recon, rk):
        ref = _smooth_hump(L, 1600, recon, rk)
        e = []
        for n in (200, 400):
            r = ref.reshape(n, -1).mean(axis=1)
            e.append(np.abs(_smooth_hump(L, n, recon, rk) - r).sum() / np.abs(r).sum())
        return e[0] / e[1]
    rw, rm = ratio(1, 3), ratio(0, 2)
    assert rw > 5.5, f"WENO/RK3 converges at ratio {rw}"
    assert rm < 4.5, f"minmod converges at ratio {rm}"


def pin_rk3_drag_factor(L=None):
    """Uniform mixture on a flat, frictionless bed, three-stage Runge-Kutta:
    v^f - v^s decays by its stability polynomial 1 - z + z^2/2 - z^3/6 per
    step (z = c_D (phi^s + alpha phi^f) dt), and rho^s q^s + rho^f q^f is
    conserved."""
    nx = ny = 6
    cd, dt, phs = 0.8, 0.1, 0.6
    p = W.default_params(c_d=cd, delta_b_deg=0.0, bc=(W.BC_TRANSMISSIVE,) * 4, rk=3)
    s = _sim(W.flat_dem(nx, ny), 5.0, 5.0, p, L)
    one = np.ones((ny, nx))
    s.set_release(2.0 * one, phs * one, 1.0 * one, 0.5 * one, 3.0 * one, -1.0 * one)
    al = p["rho_f"] / p["rho_s"]
    z = cd * (phs + al * (1 - phs)) * dt
    U0 = s.get_U()
    mix0 = p["rho_s"] * U0[1:3] + p["rho_f"] * U0[4:6]
    n = 12
    for _ in range(n):
        s.step_dt(dt)
    pr = s.primitive()
    fac = (1 - z + z * z / 2 - z ** 3 / 6) ** n
    for comp, d0 in (("x", 2.0), ("y", -1.5)):
        dv = pr[f"v{comp}_f"] - pr[f"v{comp}_s"]
        assert np.allclose(dv, d0 * fac, rtol=1e-12, atol=0), f"RK3 drag decay {dv.flat[0]} vs {d0 * fac}"
    U = s.get_U()
    mix = p["rho_s"] * U[1:3] + p["rho_f"] * U[4:6]
    assert np.allclose(mix, mix0, rtol=1e-13, atol=1e-12 * np.abs(mix0).max()), "drag not momentum-neutral"


def pin_weno_rk3_budgets_and_rotation(L=None):
    """WENO + RK3: the inflow volume balance closes (volume = time-integrated
    boundary flux + clamp volume, with the stage weights 1/6, 1/6, 2/3), a
    closed box conserves each phase's volume, and a 90-degree rotation
    commutes with the step."""
    cfg = W.inflow_config(nx=48, ny=24, dx=5.0, inlet_cells=6, recon=1, rk=3)
    s = _sim(cfg["dem"], cfg["dx"], cfg["dy"], cfg["params"], L)
    s.set_release(cfg["h"], cfg["phi_s"])
    f = cfg["inflow"]
    s.set_inflow(f["side"], f["i0"], f["i1"], f["t"], f["Q"], f["phi"])
    s.step(150)
    b = s.budget()
    for ph in ("s", "f"):
        closure = b[f"vol_{ph}"] - b[f"bnd_in_{ph}"] - b[f"clamp_{ph}"]
        assert b[f"vol_{ph}"] > 0 and abs(closure) < 1e-12 * b[f"vol_{ph}"], f"RK3 budget ({ph}): {closure}"
    n = 32
    c2 = W.release_config(nx=n, ny=n, cfl=0.2, recon=1, rk=3)
    s = _sim(c2["dem"], 5.0, 5.0, c2["params"], L)
    s.set_release(c2["h"], c2["phi_s"])
    v0 = s.budget()
    rng = np.random.default_rng(6)
    phi = rng.uniform(0.4, 0.7, (n, n))
    h = c2["h"] * (1 + 0.2 * rng.random((n, n)))
    dem = c2["dem"] + rng.random((n, n))
    a = _sim(dem, 5.0, 5.0, c2["params"], L)
    a.set_release(h, phi)
    bb = _sim(_rot(dem), 5.0, 5.0, c2["params"], L)
    bb.set_release(_rot(h), _rot(phi))
    for _ in range(25):
        dt = a.cfl_dt()
        a.step_dt(dt)
        bb.step_dt(dt)
        s.step_dt(dt)
    v1 = s.budget()
    for ph in ("s", "f"):
        assert abs(v1[f"vol_{ph}"] - v0[f"vol_{ph}"]) < 1e-13 * v0[f"vol_{ph}"], f"RK3 closed-box drift ({ph})"
    Ua, Ub = a.get_U(), bb.get_U()
    exp = np.stack([_rot(Ua[0]), -_rot(Ua[2]), _rot(Ua[1]), _rot(Ua[3]), -_rot(Ua[5]), _rot(Ua[4])])
    err = np.abs(Ub - exp).max() / np.abs(Ua).max()
    assert err < 1e-12, f"WENO/RK3 rotation invariance broken: {err}"



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


def pin_masking_reach(L=None):
    """Wet/dry masking's premise (Sect. 2.2 scheme, dry rule R5): where no cell
    within the scheme's reach holds mass, the result is exactly the zero
    state, whatever momenta the massless cells carry.  The face between two
    dry cells has zero states on both sides (minmod(0, x) = 0), so one stage
    reaches 1 cell and a two-step modified Euler step 2; the results inside the
    reach are not all zero."""
    nx, ny = 41, 33
    rng = np.random.default_rng(23)
    dem = W.spectral_dem(nx, ny, 5.0, 2.2, 40.0, seed=23) + rng.random((ny, nx))
    U = np.zeros((6, ny, nx))
    for j, i in ((3, 4), (16, 20), (30, 38), (0, 12), (20, 0)):
        U[0, j, i], U[3, j, i] = 0.9, 0.5
        U[1, j, i], U[2, j, i], U[4, j, i], U[5, j, i] = 0.9 * 1.5, -0.9 * 0.7, 0.5 * 0.4, 0.5 * 1.1
    mass = (U[0] != 0) | (U[3] != 0)
    for c in (1, 2, 4, 5):  # momenta on some massless cells: the dry rule zeroes them
        U[c] = np.where(~mass & (rng.random((ny, nx)) < 0.3), rng.normal(0.0, 1.0, (ny, nx)), U[c])
    for bc in ((0, 0, 0, 0), (1, 1, 1, 1)):
        s = _sim(dem, 5.0, 5.0, W.default_params(bc=bc), L)
        s.set_U(U)
        for r, out in ((1, s.stage(0.0, 0.02)), (2, None)):
            if out is None:
                s.set_U(U)
                s.step_dt(0.02)
                out = s.get_U()
            far = ~_dilate(mass, r)
            assert np.all(out[:, far] == 0.0), f"non-zero result beyond {r} cells of any mass (bc {bc})"
            assert np.any(out[:, ~far] != 0.0)


# ----------------------------------------------------------------------------
# internal friction: the Savage-Hutter earth-pressure coefficient (reading R10)


def _earth(params, L):
    from oracle.oracle import earth_pressure
    return earth_pressure(params, library=L)


def pin_earth_pressure_limits(L=None):
    """K_act/pass of the Savage-Hutter closure reduce to Rankine's coefficients
    (1 -/+ sin phi) / (1 +/- sin phi) on a frictionless bed (delta_b = 0), meet
    at (1 + sin^2 phi) / cos^2 phi when delta_b = phi_int, bracket 1
    (K_act < 1 < K_pass) in between, and are both 1 in the paper's form."""
    for phi in (20.0, 35.0, 41.0):
        sp = math.sin(math.radians(phi))
        ka, kp = _earth(W.default_params(k_mode=1, phi_int_deg=phi, delta_b_deg=0.0), L)
        assert abs(ka - (1 - sp) / (1 + sp)) < 1e-14 and abs(kp - (1 + sp) / (1 - sp)) < 1e-13, (phi, ka, kp)
        ka, kp = _earth(W.default_params(k_mode=1, phi_int_deg=phi, delta_b_deg=phi), L)
        lim = (1 + sp * sp) / (1 - sp * sp)
        assert abs(ka - lim) < 1e-12 and abs(kp - lim) < 1e-12, (phi, ka, kp, lim)
        ka, kp = _earth(W.default_params(k_mode=1, phi_int_deg=phi, delta_b_deg=0.6 * phi), L)
        assert ka < 1.0 < kp
    assert _earth(W.default_params(k_mode=0), L) == (1.0, 1.0)


def _solid_strip(nx, ny, dvx, dvy, seed=0, h0=2.0):
    """A wet pure-solid layer with smooth depth, moving with (vX, vY) =
    (3 + dvx i, -2 + dvy j) (dvx, dvy: velocity change per cell)."""
    rng = np.random.default_rng(seed)
    i, j = np.meshgrid(np.arange(nx), np.arange(ny))
    h = h0 + 0.3 * np.sin(0.4 * i + 0.3 * j) + 0.1 * rng.random((ny, nx))
    return h, 3.0 + dvx * i, -2.0 + dvy * j


def _stage_interior(dem, params, h, vx, vy, L, dt=0.05):
    s = _sim(dem, 5.0, 5.0, params, L)
    s.set_release(h, np.ones_like(h), vx, vy)
    return s.stage(0.0, dt)[:, 2:-2, 2:-2]


def pin_earth_pressure_regimes(L=None):
    """One stage of a pure solid (rho_f = 0, no fluid) whose velocity grows
    across every face (stretching) equals the paper's stage with eps scaled by
    K_act -- eps enters a pure solid's step only through its pressure and
    celerity -- and with a velocity that falls across every face
    (compression) the one with eps scaled by K_pass; each axis chooses by its
    own velocity component (an x-strip that compresses in X while its Y
    velocity grows is passive, and the y-strip likewise); a face next to a
    cell without solid is active."""
    dem = W.incline_dem(24, 20, 5.0, 5.0, 15.0) + 0.5 * W.incline_dem(24, 20, 5.0, 5.0, 10.0, axis="y")
    base = _pure_solid(k_mode=1, phi_int_deg=35.0, delta_b_deg=25.0, bc=(W.BC_TRANSMISSIVE,) * 4)
    ka, kp = _earth(base, L)
    k0 = dict(base, k_mode=0)
    for dv, K in ((0.05, ka), (-0.05, kp)):
        h, vx, vy = _solid_strip(24, 20, dv, dv)
        got = _stage_interior(dem, base, h, vx, vy, L)
        ref = _stage_interior(dem, dict(k0, eps=K), h, vx, vy, L)
        assert np.allclose(got[:3], ref[:3], rtol=1e-12, atol=1e-12 * np.abs(ref[:3]).max()), (dv, K)
        plain = _stage_interior(dem, k0, h, vx, vy, L)
        assert np.abs(got[1:3] - plain[1:3]).max() > 1e-6 * np.abs(plain[1:3]).max(), "K has no effect"
    # each axis by its own component: 1-cell-wide strips
    for nx, ny, dvx, dvy in ((30, 1, -0.05, 0.05), (1, 30, 0.05, -0.05)):
        demk = W.incline_dem(nx, ny, 5.0, 5.0, 12.0)
        h, vx, vy = _solid_strip(nx, ny, dvx, dvy)
        sl = (slice(None), slice(2, -2), slice(None)) if nx == 1 else (slice(None), slice(None), slice(2, -2))
        s1 = _sim(demk, 5.0, 5.0, base, L)
        s1.set_release(h, np.ones_like(h), vx, vy)
        s2 = _sim(demk, 5.0, 5.0, dict(k0, eps=kp), L)
        s2.set_release(h, np.ones_like(h), vx, vy)
        got, ref = s1.stage(0.0, 0.05)[sl], s2.stage(0.0, 0.05)[sl]
        assert np.allclose(got[:3], ref[:3], rtol=1e-12, atol=1e-12 * np.abs(ref[:3]).max()), (nx, ny)
    # isolated solid cells moving fast: every face borders a cell without solid
    # (empty, or a film thinner than h_dry whose momentum would, if counted,
    # make the cell's velocity fall across it)
    nx = ny = 12
    h = np.zeros((ny, nx))
    h[3, 3] = h[8, 7] = 1.5
    vx = np.full((ny, nx), 4.0)
    vy = np.full((ny, nx), -3.0)
    h[8, 6] = h[8, 8] = h[7, 7] = h[9, 7] = 0.5 * base["h_dry"]
    vx[8, 6], vx[8, 8], vy[7, 7], vy[9, 7] = 20.0, -20.0, 20.0, -20.0
    flat = W.flat_dem(nx, ny)
    got = _stage_interior(flat, base, h, vx, vy, L)
    ref = _stage_interior(flat, dict(k0, eps=ka), h, vx, vy, L)
    assert np.allclose(got[:3], ref[:3], rtol=1e-12, atol=1e-12 * np.abs(ref[:3]).max()), "dry neighbour"


def pin_earth_pressure_fluid_unaffected(L=None):
    """K belongs to the solid: in one stage of a two-phase mixture the fluid
    components are the same in both forms, bit for bit."""
    cfg = W.release_config(nx=20, ny=18, cfl=0.2)
    st = W.random_state(20, 18, seed=4, dry_frac=0.0)
    out = []
    for km in (0, 1):
        s = _sim(cfg["dem"], 5.0, 5.0, dict(cfg["params"], k_mode=km), L)
        s.set_release(st["h"], st["phi_s"], st["vx_s"], st["vy_s"], st["vx_f"], st["vy_f"])
        out.append(s.stage(0.0, 0.02))
    assert np.array_equal(out[0][3:], out[1][3:]), "the earth pressure touched the fluid"
    assert not np.array_equal(out[0][:3], out[1][:3])


def pin_earth_pressure_wave_speed(L=None):
    """The CFL wave speed of a pure solid at rest on a flat bed is
    sqrt(K_pass g h) with the earth-pressure option (the larger coefficient
    bounds the celerity in either regime)."""
    nx, ny = 5, 4
    one = np.ones((ny, nx))
    p = _pure_solid(k_mode=1, phi_int_deg=35.0, delta_b_deg=25.0)
    s = _sim(W.flat_dem(nx, ny), 5.0, 5.0, p, L)
    s.set_release(3.0 * one, one)
    _, kp = _earth(p, L)
    assert abs(s.max_speed() - math.sqrt(kp * G * 3.0)) < 1e-13


def _sh_k_reference(t_end, H0, L0, zeta, delta, K, u0=0.0, w0=0.0):
    """Centre travel and half-length of the parabolic cap with earth-pressure
    coefficient K: s_c'' = g (sin z - tan d cos z) with s_c'(0) = u0, and
    L'' = 2 K g cos z H0 L0 / L^2 with L'(0) = w0 (RK4, fine steps)."""
    a = G * (math.sin(zeta) - math.tan(delta) * math.cos(zeta))
    k = 2 * K * G * math.cos(zeta) * H0 * L0

    def f(y):
        return np.array([y[1], k / y[0] ** 2])

    y = np.array([L0, w0])
    n = 20000
    h = t_end / n
    for _ in range(n):
        k1 = f(y)
        k2 = f(y + 0.5 * h * k1)
        k3 = f(y + 0.5 * h * k2)
        k4 = f(y + h * k3)
        y = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return u0 * t_end + 0.5 * a * t_end ** 2, y[0], y[1]


def _cap_moments(s, x, zeta):
    U1 = s.get_U()[0, 0]
    sc = x / math.cos(zeta)
    m = U1.sum()
    c = (sc * U1).sum() / m
    return c, math.sqrt(5 * ((sc - c) ** 2 * U1).sum() / m)


def pin_savage_hutter_earth_pressure(L=None):
    """The parabolic cap with internal friction (Savage-Hutter, K != 1), pure
    solid on a 35 degree plane, delta_b = 25, phi_int = 35 degrees, launched
    downslope with a linear velocity field along the slope, every point
    moving downslope: spreading, every cell is active and the half-length
    follows L'' = 2 K_act g cos z H0 L0 / L^2; converging, every cell is
    passive (K_pass) until the cap turns.  The centre follows
    s_c'' = g (sin z - tan d cos z) in both.  Each half-length is held
    closer to its own coefficient's solution than a quarter of the distance
    to the other regime's (K = 1 for the active case)."""
    zeta, delta = math.radians(35.0), math.radians(25.0)
    H0, L0, dx = 5.0, 100.0, 1.0
    nx = 1400
    x = (np.arange(nx) + 0.5) * dx
    X0 = 200.0
    p = _pure_solid(delta_b_deg=25.0, phi_int_deg=35.0, k_mode=1, cfl=0.1)
    ka, kp = _earth(p, L)
    h = H0 * np.clip(1 - ((x - X0) / (L0 * math.cos(zeta))) ** 2, 0, None)
    dem = W.incline_dem(nx, 1, dx, dx, 35.0)
    sc0 = X0 / math.cos(zeta)
    for u0, w0, t_end, K, K_other in ((12.0, 5.0, 4.0, ka, 1.0), (15.0, -10.0, 1.5, kp, ka)):
        # velocity along the slope u0 + (s - s_c) w0 / L0, as its horizontal projection
        v = (u0 + (x / math.cos(zeta) - sc0) * w0 / L0) * math.cos(zeta)
        s = _sim(dem, dx, dx, p, L)
        s.set_release(h[None, :], np.ones((1, nx)), v[None, :], None)
        while s.t < t_end:
            s.step(5)
        ds_ref, L_ref, w = _sh_k_reference(s.t, H0, L0, zeta, delta, K, u0, w0)
        _, L_other, _ = _sh_k_reference(s.t, H0, L0, zeta, delta, K_other, u0, w0)
        assert w * w0 > 0, "the reference cap turned within the window"
        c, Lnum = _cap_moments(s, x, zeta)
        ds = c - sc0
        assert abs(ds - ds_ref) / ds_ref < 5e-3, f"SH-K centre travel {ds} vs {ds_ref} (w0 {w0})"
        assert abs(Lnum - L_ref) < 0.25 * abs(L_ref - L_other), \
            f"SH-K half-length {Lnum} vs {L_ref} (K {K}; {L_other} with K {K_other})"


def pin_rotation_earth_pressure(L=None, steps=30):
    """90 degree rotation invariance with the earth-pressure option (each axis
    chooses its coefficient by its own velocity component)."""
    n = 32
    cfg = W.release_config(nx=n, ny=n, cfl=0.2)
    p = dict(cfg["params"], k_mode=1)
    rng = np.random.default_rng(8)
    phi = rng.uniform(0.4, 0.7, (n, n))
    h = cfg["h"] * (1 + 0.2 * rng.random((n, n)))
    dem = cfg["dem"] + rng.random((n, n))
    a = _sim(dem, 5.0, 5.0, p, L)
    a.set_release(h, phi)
    b = _sim(_rot(dem), 5.0, 5.0, p, L)
    b.set_release(_rot(h), _rot(phi))
    for _ in range(steps):
        dt = a.cfl_dt()
        assert abs(dt - b.cfl_dt()) <= 1e-14 * dt, "rotated run takes a different dt"
        a.step_dt(dt)
        b.step_dt(dt)
    Ua, Ub = a.get_U(), b.get_U()
    exp = np.stack([_rot(Ua[0]), -_rot(Ua[2]), _rot(Ua[1]), _rot(Ua[3]), -_rot(Ua[5]), _rot(Ua[4])])
    err = np.abs(Ub - exp).max() / np.abs(Ua).max()
    assert err < 1e-12, f"rotation invariance broken with k_mode 1: {err}"


ALL_PINS = [
    # cheap pins first: the planted-mistake harness stops at the first pin that fails
    pin_masking_reach, pin_inflow_every_side, pin_stage_times, pin_time_step_cap, pin_positivity_clamp,
    pin_rotation_transmissive, pin_rotation_rectangular, pin_rotation_viscous, pin_max_speed_everywhere,
    pin_plane_equilibrium_eps, pin_lake_curved_bed_residual_converges, pin_step_composition, pin_phase_symmetry, pin_inflow_mirror,
    pin_uniform_flow_viscous, pin_thin_film_has_no_velocity, pin_clamp_count,
    pin_viscous_only_where_the_fluid_is_wet, pin_thin_cell_has_no_phase_fractions, pin_budget_sums,
    pin_friction_buoyant, pin_step_clock, pin_max_speed_rows, pin_step_amax, pin_drag_neutral_on_a_slope,
    pin_geometry_plane, pin_curvature, pin_conservation_closed, pin_lake_flat, pin_lake_plane,
    pin_mixture_plane_rest, pin_mixture_no_separation, pin_heap_rest, pin_ritter, pin_savage_hutter, pin_drag,
    pin_wave_speed, pin_rotation, pin_inflow, pin_friction, pin_closed_box, pin_viscous, pin_fluid_friction,
    pin_cu_upwind_dependence, pin_cu_conservation_and_ritter, pin_cu_rotation,
    pin_weno_linear_exact, pin_weno_rk3_dam_break, pin_weno_smooth_order, pin_rk3_drag_factor,
    pin_weno_rk3_budgets_and_rotation,
    pin_earth_pressure_limits, pin_earth_pressure_regimes, pin_earth_pressure_fluid_unaffected,
    pin_earth_pressure_wave_speed, pin_savage_hutter_earth_pressure, pin_rotation_earth_pressure]
