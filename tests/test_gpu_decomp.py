"""Row-strip domain decomposition on the GPU: strips (moses.Sim with owned
rows, through the C-ABI) in one process on one GPU, their overlap rows
exchanged by device copies (moses_get_rows_device / moses_set_rows_device)
and the CFL maximum agreed on the host (moses_set_max_speed).  The strips'
own rows must equal the undecomposed GPU run bit for bit in both precisions,
every tile shape, the three-stage Runge-Kutta step, the earth-pressure form
and a west-side inflow, and (FP64) the oracle within 1e-10.  The strips run
one after another on one stream: no kernel waits on another strip's.
"""
import numpy as np
import pytest

from oracle.oracle import from_config as oracle_from_config
from paper_2104_06784_gb300 import decomp as D
from paper_2104_06784_gb300 import moses, workloads as W
from tests.test_decomp_cpu import _dense, _spectral
from tests.test_gpu_parity import TOL64, rel_maxnorm

pytestmark = pytest.mark.gpu


def _strips(cfg, world, precision, tile=None):
    o = D.overlap_rows(cfg["params"])
    strips = [D.GpuStrip(cfg, p, precision=precision) for p in D.plan(cfg["dem"].shape[0], world, o)]
    if tile is not None:
        for s in strips:
            s.sim.set_tile(tile)
    return strips


def _own(strips):
    return np.concatenate([s.own_state() for s in strips], axis=1)


def _whole(cfg, precision, n, tile=None):
    g = moses.from_config(cfg, precision=precision)
    if tile is not None:
        g.set_tile(tile)
    g.step(n)
    return g


@pytest.mark.parametrize("precision", [moses.FP64, moses.FP32])
@pytest.mark.parametrize("world", [2, 3, 4])
@pytest.mark.parametrize("bc", [0, 1])
def test_strips_equal_the_whole_domain_bit_for_bit(precision, world, bc):
    cfg = _spectral(bc=bc)
    n = 40
    strips = _strips(cfg, world, precision)
    D.LocalComm(strips).run(n)
    g = _whole(cfg, precision, n)
    U = g.get_conserved()
    assert np.array_equal(_own(strips), U)
    t = g.budget()["t"]
    assert all(s.sim.budget()["t"] == t for s in strips)
    assert any(U[0, s.p.own1 - 1].any() and U[0, s.p.own1].any() for s in strips[:-1])
    if precision == moses.FP64:
        o = oracle_from_config(cfg)
        o.step(n)
        assert rel_maxnorm(_own(strips), o.get_U()) < TOL64


@pytest.mark.parametrize("tile", [0, 1, 2, 3])
def test_every_tile_shape(tile):
    cfg = _spectral()
    strips = _strips(cfg, 3, moses.FP64, tile)
    D.LocalComm(strips).run(25)
    assert np.array_equal(_own(strips), _whole(cfg, moses.FP64, 25, tile).get_conserved())


@pytest.mark.parametrize("over", [dict(rk=3), dict(k_mode=1)], ids=["rk3", "earth_pressure"])
@pytest.mark.parametrize("precision", [moses.FP64, moses.FP32])
def test_runge_kutta_and_earth_pressure(over, precision):
    cfg = _spectral(**over)
    strips = _strips(cfg, 4, precision)
    D.LocalComm(strips).run(25)
    assert np.array_equal(_own(strips), _whole(cfg, precision, 25).get_conserved())


def test_dense_state_and_west_inflow():
    for cfg, world, n in ((_dense(2), 4, 15), (W.inflow_config(nx=48, ny=90, inlet_cells=6, cfl=0.3), 3, 60)):
        for precision in (moses.FP64, moses.FP32):
            strips = _strips(cfg, world, precision)
            D.LocalComm(strips).run(n)
            U = _whole(cfg, precision, n).get_conserved()
            assert np.count_nonzero(U[0]) > 0
            assert np.array_equal(_own(strips), U), (cfg["name"], precision)


def test_budgets_add_up_over_the_strips():
    """Each strip's budget counts its own rows: the volumes and the boundary
    inflow of all strips add up to the whole domain's (FP64 sums in another
    order: 1e-12 relative)."""
    cfg = W.inflow_config(nx=48, ny=90, inlet_cells=6, cfl=0.3)
    strips = _strips(cfg, 3, moses.FP64)
    D.LocalComm(strips).run(80)
    b = _whole(cfg, moses.FP64, 80).budget()
    for k in ("vol_s", "vol_f", "bnd_in_s", "bnd_in_f"):
        tot = sum(s.sim.budget()[k] for s in strips)
        assert abs(tot - b[k]) <= 1e-12 * max(abs(b[k]), 1e-30), (k, tot, b[k])
    assert b["bnd_in_s"] > 0


def test_strip_calls_validate_and_strips_join_no_batch_or_adjoint():
    cfg = _spectral()
    s = _strips(cfg, 2, moses.FP64)[0]
    with pytest.raises(moses.MosesError):
        s.sim.set_owned_rows(5, 5)
    with pytest.raises(moses.MosesError):
        s.sim.set_max_speed(float("nan"))
    with pytest.raises(moses.MosesError):
        s.sim.get_rows_device(s.sim.ny - 1, 2, 0)
    with pytest.raises(moses.MosesError):
        moses.Batch([s.sim])
    with pytest.raises(moses.MosesError):
        s.sim.adjoint_misfit(2, np.zeros((s.sim.ny, s.sim.nx)))
    assert s.sim.row_planes == 6
    assert _strips(cfg, 2, moses.FP32)[0].sim.row_planes == 8
