"""Adjoint of the two-phase step (moses_stage_adjoint, moses_adjoint_misfit).

Stage level: <lam, (S(U + e v) - S(U - e v)) / 2e> = <S'(U)^T lam, v> on wet
random states (the dot-product test), for closed, transmissive and mixed
boundaries and an inflow segment.  Run level: gradients of the deposit misfit
with respect to the basal friction angle, the drag coefficient and the release
thickness against FP64 central differences of the CPU oracle rerun with the
same (frozen) time-step sequence, on small instances whose finite differences
are consistent at two step sizes (no kink crossed).
"""
import numpy as np
import pytest

from oracle.oracle import OracleSim, from_config as oracle_from_config
from paper_2104_06784_gb300 import moses, workloads as W

pytestmark = pytest.mark.gpu


def _wet_state(nx, ny, seed):
    rng = np.random.default_rng(seed)
    return dict(h=0.5 + 2.0 * rng.random((ny, nx)), phi_s=rng.uniform(0.3, 0.8, (ny, nx)),
                vx_s=rng.standard_normal((ny, nx)), vy_s=rng.standard_normal((ny, nx)),
                vx_f=rng.standard_normal((ny, nx)), vy_f=rng.standard_normal((ny, nx)))


def _stage_sim(nx, ny, bc, inflow, prec, seed, k_mode=0):
    if inflow:
        cfg = W.inflow_config(nx=nx, ny=ny, dx=5.0, inlet_cells=6, k_mode=k_mode)
        g = moses.Sim(cfg["dem"], 5.0, 5.0, cfg["params"], precision=prec)
        f = cfg["inflow"]
        g.set_inflow(f["side"], f["i0"], f["i1"], f["t"], f["Q"], f["phi"])
    else:
        dem = W.spectral_dem(nx, ny, 5.0, 2.2, 30.0, seed=seed, band_m=40.0)
        g = moses.Sim(dem, 5.0, 5.0, W.default_params(bc=bc, c_d=0.05, k_mode=k_mode), precision=prec)
    st = _wet_state(nx, ny, seed)
    g.set_release(st["h"], st["phi_s"], st["vx_s"], st["vy_s"], st["vx_f"], st["vy_f"])
    return g


@pytest.mark.parametrize("k_mode", [0, 1])
@pytest.mark.parametrize("nx,ny,bc,inflow", [(45, 37, (0, 0, 0, 0), False), (70, 20, (1, 1, 1, 1), False),
                                             (33, 41, (0, 1, 1, 0), False), (60, 30, (1, 1, 1, 1), True)])
def test_stage_adjoint_dot_product(nx, ny, bc, inflow, k_mode):
    g = _stage_sim(nx, ny, bc, inflow, moses.FP64, seed=1, k_mode=k_mode)
    U = g.get_conserved()
    rng = np.random.default_rng(101)
    lam = rng.standard_normal(U.shape)
    v = rng.standard_normal(U.shape) * np.abs(U).reshape(6, -1).max(axis=1)[:, None, None]
    t, dt, eps = 30.0, 0.01, 1e-6
    li, _ = g.stage_adjoint(t, dt, lam)
    g.set_conserved(U + eps * v)
    Sp = g.stage(t, dt)
    g.set_conserved(U - eps * v)
    Sm = g.stage(t, dt)
    fd = (lam * (Sp - Sm)).sum() / (2 * eps)
    ad = (li * v).sum()
    assert abs(fd - ad) <= 1e-7 * abs(fd), (fd, ad)


@pytest.mark.parametrize("k_mode", [0, 1])
@pytest.mark.parametrize("nx,ny,bc,inflow", [(45, 37, (0, 0, 0, 0), False), (70, 20, (1, 1, 1, 1), False),
                                             (60, 30, (1, 1, 1, 1), True)])
def test_stage_adjoint_dot_product_richardson(nx, ny, bc, inflow, k_mode):
    """The dot-product test against a sharper difference quotient: central
    differences at two step sizes extrapolated (Richardson, error O(e^4)), so
    that the bar is set by the FP64 rounding of the forward stage (relative
    noise about 1e-16 / e) rather than by the truncation error: 1e-9."""
    g = _stage_sim(nx, ny, bc, inflow, moses.FP64, seed=3, k_mode=k_mode)
    U = g.get_conserved()
    rng = np.random.default_rng(202)
    lam = rng.standard_normal(U.shape)
    v = rng.standard_normal(U.shape) * np.abs(U).reshape(6, -1).max(axis=1)[:, None, None]
    t, dt = 30.0, 0.01
    li, _ = g.stage_adjoint(t, dt, lam)
    ad = (li * v).sum()

    def quotient(eps):
        g.set_conserved(U + eps * v)
        Sp = g.stage(t, dt)
        g.set_conserved(U - eps * v)
        Sm = g.stage(t, dt)
        return (lam * (Sp - Sm)).sum() / (2 * eps)

    d1, d2 = quotient(2e-6), quotient(1e-6)
    rich = (4 * d2 - d1) / 3
    assert abs(rich - ad) <= 1e-9 * abs(rich), (rich, ad, d1, d2)


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 1, 1)])
def test_stage_adjoint_dot_product_sparse(bc):
    """Wet blobs on tile edges in a dry domain: the dry tiles skip their face
    terms (wet/dry masking) and their neighbours read the mass-only adjoints
    of the dry cells.  Dot-product test with lam everywhere and v on the wet
    cells (the stage is differentiable there), central differences."""
    nx, ny = 97, 41
    dem = W.spectral_dem(nx, ny, 5.0, 2.2, 30.0, seed=4, band_m=40.0)
    g = moses.Sim(dem, 5.0, 5.0, W.default_params(bc=bc, c_d=0.05))
    rng = np.random.default_rng(17)
    h = np.zeros((ny, nx))
    for j0, i0 in ((6, 29), (15, 62), (30, 0), (0, 90), (23, 45)):
        h[j0:j0 + 3, i0:i0 + 4] = 0.8 + rng.random((min(3, ny - j0), min(4, nx - i0)))
    st = _wet_state(nx, ny, 5)
    g.set_release(h, st["phi_s"], st["vx_s"], st["vy_s"], st["vx_f"], st["vy_f"])
    U = g.get_conserved()
    lam = rng.standard_normal(U.shape)
    v = rng.standard_normal(U.shape) * np.abs(U).reshape(6, -1).max(axis=1)[:, None, None] * (h > 0)[None]
    t, dt, eps = 0.0, 0.005, 1e-6
    li, _ = g.stage_adjoint(t, dt, lam)
    g.set_conserved(U + eps * v)
    Sp = g.stage(t, dt)
    g.set_conserved(U - eps * v)
    Sm = g.stage(t, dt)
    fd = (lam * (Sp - Sm)).sum() / (2 * eps)
    ad = (li * v).sum()
    assert abs(fd - ad) <= 1e-7 * abs(fd), (fd, ad)
    # on cells at least 3 away from any mass the stage is the identity on the
    # masses and zeroes the momenta: so is its adjoint there
    far = np.ones((ny, nx), bool)
    wet = h > 0
    for dj in range(-3, 4):
        for di in range(-3, 4):
            far &= ~np.roll(np.roll(wet, dj, 0), di, 1) | _rolled_out(ny, nx, dj, di)
    assert far.sum() > 0.5 * nx * ny
    assert np.array_equal(li[0][far], lam[0][far]) and np.array_equal(li[3][far], lam[3][far])
    for c in (1, 2, 4, 5):
        assert not li[c][far].any()


def _rolled_out(ny, nx, dj, di):
    """Cells whose np.roll source wrapped around the grid edge (not neighbours)."""
    m = np.zeros((ny, nx), bool)
    if dj > 0:
        m[:dj, :] = True
    elif dj < 0:
        m[dj:, :] = True
    if di > 0:
        m[:, :di] = True
    elif di < 0:
        m[:, di:] = True
    return m


@pytest.mark.parametrize("k_mode", [0, 1])
def test_stage_adjoint_parameter_partials(k_mode):
    """lam . dS/d tan(delta_b), lam . dS/d c_D and (k_mode 1) lam . dS/d phi_int
    against central differences of the stage."""
    nx, ny = 40, 30
    dem = W.spectral_dem(nx, ny, 5.0, 2.2, 30.0, seed=3, band_m=40.0)
    st = _wet_state(nx, ny, 3)
    rng = np.random.default_rng(7)
    lam = rng.standard_normal((6, ny, nx))
    t, dt = 0.0, 0.01

    def stage(delta_deg, c_d, phi_deg=35.0):
        g = moses.Sim(dem, 5.0, 5.0, W.default_params(delta_b_deg=delta_deg, c_d=c_d, bc=(1, 1, 1, 1), k_mode=k_mode,
                                                      phi_int_deg=phi_deg))
        g.set_release(st["h"], st["phi_s"], st["vx_s"], st["vy_s"], st["vx_f"], st["vy_f"])
        return g, g.stage(t, dt)

    g, _ = stage(25.0, 0.05)
    _, gp = g.stage_adjoint(t, dt, lam)
    h = 1e-6
    tp, tm = np.tan(np.radians(25.0)) + h, np.tan(np.radians(25.0)) - h
    fd_tan = (lam * (stage(np.degrees(np.arctan(tp)), 0.05)[1] - stage(np.degrees(np.arctan(tm)), 0.05)[1])).sum() / (2 * h)
    fd_cd = (lam * (stage(25.0, 0.05 + 1e-7)[1] - stage(25.0, 0.05 - 1e-7)[1])).sum() / 2e-7
    assert abs(gp[0] - fd_tan) <= 1e-6 * abs(fd_tan), (gp[0], fd_tan)
    assert abs(gp[1] - fd_cd) <= 1e-6 * abs(fd_cd), (gp[1], fd_cd)
    if k_mode == 0:
        assert gp[2] == 0.0
        return
    fd_phi = (lam * (stage(25.0, 0.05, 35.0 + np.degrees(h))[1] - stage(25.0, 0.05, 35.0 - np.degrees(h))[1])).sum() / (2 * h)
    assert gp[2] != 0.0 and abs(gp[2] - fd_phi) <= 1e-6 * abs(fd_phi), (gp[2], fd_phi)


def test_stage_adjoint_fp32_tracks_fp64():
    g64 = _stage_sim(45, 37, (0, 0, 0, 0), False, moses.FP64, seed=2)
    g32 = _stage_sim(45, 37, (0, 0, 0, 0), False, moses.FP32, seed=2)
    lam = np.random.default_rng(9).standard_normal((6, 37, 45))
    l64, _ = g64.stage_adjoint(30.0, 0.01, lam)
    l32, _ = g32.stage_adjoint(30.0, 0.01, lam)
    assert np.abs(l32 - l64).sum() <= 1e-5 * np.abs(l64).sum()


# ----------------------------------------------------------------------------
# deposit misfit over many steps


def _misfit_setup(cfg, N, hidden=dict(delta_b_deg=22.0, c_d=3e-3)):
    ct = dict(cfg)
    ct["params"] = dict(cfg["params"], **hidden)
    gt = moses.from_config(ct)
    gt.step(N)
    J = oracle_from_config(cfg).geometry()["J"]
    hs_t = gt.get_conserved()[0] / J
    g = moses.from_config(cfg)
    dts = []
    for _ in range(N):
        dts.append(g.next_dt()[0])
        g.step(1)
    return hs_t, J, dts


def _oracle_loss(cfg, params, dts, hs_t, J, h0=None):
    o = OracleSim(cfg["dem"], cfg["dx"], cfg["dy"], params)
    o.set_release(cfg["h"] if h0 is None else h0, cfg["phi_s"])
    if cfg.get("inflow"):
        f = cfg["inflow"]
        o.set_inflow(f["side"], f["i0"], f["i1"], f["t"], f["Q"], f["phi"])
    for dt in dts:
        o.step_dt(dt)
    hs = o.get_U()[0] / J
    return float(((hs - hs_t) ** 2).sum() * cfg["dx"] * cfg["dy"])


@pytest.mark.parametrize("case,k_mode", [("spectral64", 0), ("arc", 0), ("inflow", 0), ("wet65", 0),
                                         ("spectral64", 1), ("arc", 1)])
def test_misfit_gradient_matches_fp64_central_differences(case, k_mode):
    """With k_mode 1 also the internal friction angle, which enters through
    the Savage-Hutter coefficients (and delta_b through them besides tan)."""
    if case == "spectral64":
        cfg, N, C = W.large_release_config(n=64, dx=5.0, seed=7, volume=2.5e4, radius_cells=6, k_mode=k_mode), 80, 9
    elif case == "arc":
        # a pile centred on a cell column stays mirror-symmetric, and across the
        # axis the two x-momentum differences are equal: minmod is at a tie,
        # where the step is not differentiable.  The pile is moved off the axis.
        cfg, N, C = W.release_config(nx=48, ny=64, cfl=0.2, k_mode=k_mode), 60, 7
        cfg["h"] = W.parabolic_cap(48, 64, 5.0, 5.0, 24.37, 63 - 30 * 64 // 128, 20 * 48 / 128, 5.0)
    elif case == "wet65":
        # a layer on every cell against closed walls, on a grid whose last tile
        # column holds one cell (65 = 2 x 32 + 1): the ghost adjoints are
        # folded by their own launch, and the walls take part
        cfg, N, C = W.large_release_config(n=65, ny=49, dx=5.0, seed=11, volume=2e4, radius_cells=5,
                                           bc=(0, 0, 0, 0)), 80, 9
        cfg["h"] = cfg["h"] + 0.3
    else:  # material enters through a hydrograph: the recompute must see the same times
        cfg, N, C = W.inflow_config(nx=48, ny=32, dx=5.0, inlet_cells=6), 120, 11
    hs_t, J, dts = _misfit_setup(cfg, N)
    g = moses.from_config(cfg)
    r = g.adjoint_misfit(N, hs_t, ckpt_every=C, release_phi=cfg["phi_s"])
    p0 = cfg["params"]
    assert abs(r["loss"] - _oracle_loss(cfg, p0, dts, hs_t, J)) <= 1e-10 * r["loss"]
    # small steps: the FP64 rounding noise of L (~1e-16 L / step) stays far
    # below the tolerance while the chance of crossing a kink (a cell reaching
    # the dry threshold or the stopping condition) shrinks with the step; two
    # step sizes must agree, which shows that no kink was crossed
    params = [("delta_b_deg", 0, 1e-5), ("c_d", 2, 1e-8)] + ([("phi_int_deg", 1, 1e-5)] if k_mode == 1 else [])
    for name, idx, h in params:
        fd = [(_oracle_loss(cfg, dict(p0, **{name: p0[name] + s}), dts, hs_t, J)
               - _oracle_loss(cfg, dict(p0, **{name: p0[name] - s}), dts, hs_t, J)) / (2 * s) for s in (h, h / 2)]
        assert fd[1] != 0.0 and abs(fd[0] - fd[1]) <= 2e-6 * abs(fd[0]), (name, "finite differences cross a kink", fd)
        assert abs(r["g_params"][idx] - fd[1]) <= 1e-5 * abs(fd[1]), (name, r["g_params"][idx], fd)
    if k_mode == 0:
        assert r["g_params"][1] == 0.0
    if case in ("inflow", "wet65"):
        return
    # release thickness: directional derivative along a relative perturbation
    # of the pile.  It moves the wet front, where a cell that crosses the dry
    # threshold within the step puts a jump into L; three step sizes whose
    # differences agree to 1e-6 show that none did, and the adjoint must then
    # meet them at the tolerance of the other gradients.
    v = np.random.default_rng(5).standard_normal(cfg["h"].shape) * cfg["h"]
    steps = (1e-7, 3e-8, 1e-8) if k_mode == 1 else (1e-6, 1e-7, 1e-8)
    fdh = [(_oracle_loss(cfg, p0, dts, hs_t, J, cfg["h"] + s * v) - _oracle_loss(cfg, p0, dts, hs_t, J, cfg["h"] - s * v))
           / (2 * s) for s in steps]
    adh = float((r["g_release_h"] * v).sum())
    for a, b in ((0, 1), (1, 2)):
        assert abs(fdh[a] - fdh[b]) <= 1e-6 * abs(fdh[a]), ("finite differences cross a kink", adh, fdh)
    assert abs(adh - fdh[1]) <= 1e-5 * abs(fdh[1]), (adh, fdh)


def test_misfit_gradient_does_not_depend_on_checkpoint_interval():
    cfg = W.large_release_config(n=64, dx=5.0, seed=7, volume=2.5e4, radius_cells=6)
    hs_t, _, _ = _misfit_setup(cfg, 40)
    res = [moses.from_config(cfg).adjoint_misfit(40, hs_t, ckpt_every=C) for C in (1, 6, 40)]
    for r in res[1:]:
        assert abs(r["loss"] - res[0]["loss"]) <= 1e-14 * res[0]["loss"]  # loss sum order varies
        assert np.allclose(r["g_params"], res[0]["g_params"], rtol=1e-12, atol=0)
        assert np.allclose(r["g_release_h"], res[0]["g_release_h"], rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("k_mode", [0, 1])
def test_misfit_fp32_gradient_tracks_fp64(k_mode):
    cfg = W.large_release_config(n=64, dx=5.0, seed=7, volume=2.5e4, radius_cells=6, k_mode=k_mode)
    hs_t, _, _ = _misfit_setup(cfg, 80)
    r64 = moses.from_config(cfg).adjoint_misfit(80, hs_t, ckpt_every=9)
    r32 = moses.from_config(cfg, precision=moses.FP32).adjoint_misfit(80, hs_t, ckpt_every=9)
    for idx in ((0, 1, 2) if k_mode else (0, 2)):
        assert abs(r32["g_params"][idx] - r64["g_params"][idx]) <= 1e-3 * abs(r64["g_params"][idx])


def test_autograd_function():
    torch = pytest.importorskip("torch")
    cfg = W.large_release_config(n=64, dx=5.0, seed=7, volume=2.5e4, radius_cells=6)
    hs_t, _, _ = _misfit_setup(cfg, 40)
    h0 = torch.tensor(cfg["h"], dtype=torch.float64, requires_grad=True)
    db = torch.tensor(25.0, dtype=torch.float64, requires_grad=True)
    cd = torch.tensor(1e-3, dtype=torch.float64, requires_grad=True)
    pi = torch.tensor(35.0, dtype=torch.float64, requires_grad=True)
    loss = moses.deposit_misfit(cfg, h0, db, cd, pi, hs_t, 40, precision=moses.FP64)
    (2.0 * loss).backward()
    r = moses.from_config(cfg).adjoint_misfit(40, hs_t, release_phi=cfg["phi_s"])
    assert abs(float(loss) - r["loss"]) <= 1e-12 * r["loss"]
    assert abs(float(db.grad) - 2 * r["g_params"][0]) <= 1e-12 * abs(r["g_params"][0])
    assert abs(float(cd.grad) - 2 * r["g_params"][2]) <= 1e-12 * abs(r["g_params"][2])
    assert float(pi.grad) == 0.0
    assert np.allclose(h0.grad.numpy(), 2 * r["g_release_h"], rtol=1e-12, atol=0)


def test_autograd_function_internal_friction():
    """With the earth-pressure option the internal friction angle has a
    gradient, and the autograd.Function passes it through."""
    torch = pytest.importorskip("torch")
    cfg = W.large_release_config(n=64, dx=5.0, seed=7, volume=2.5e4, radius_cells=6, k_mode=1)
    hs_t, _, _ = _misfit_setup(cfg, 40)
    h0 = torch.tensor(cfg["h"], dtype=torch.float64, requires_grad=True)
    db = torch.tensor(25.0, dtype=torch.float64, requires_grad=True)
    cd = torch.tensor(1e-3, dtype=torch.float64, requires_grad=True)
    pi = torch.tensor(35.0, dtype=torch.float64, requires_grad=True)
    loss = moses.deposit_misfit(cfg, h0, db, cd, pi, hs_t, 40, precision=moses.FP64)
    loss.backward()
    r = moses.from_config(cfg).adjoint_misfit(40, hs_t, release_phi=cfg["phi_s"])
    assert r["g_params"][1] != 0.0
    assert abs(float(pi.grad) - r["g_params"][1]) <= 1e-12 * abs(r["g_params"][1])
    assert abs(float(db.grad) - r["g_params"][0]) <= 1e-12 * abs(r["g_params"][0])
