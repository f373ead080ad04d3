"""Row-strip domain decomposition on CPU ranks, with the FP64 oracle as each
strip's engine (no GPU).

Each strip steps its window (own rows plus 2 x stages + 1 rows of overlap)
with the CFL maximum agreed over all strips, then takes its neighbours' own
rows into its overlap.  The own rows must then equal the undecomposed
oracle's, bit for bit, step after step: the decomposition changes where a
cell is computed, never what it sees.  In-process strips (LocalComm) cover
several splits, both boundary kinds, the three-stage Runge-Kutta step and a
west-side inflow; two gloo processes (TorchComm over torch.distributed)
cover the exchange over a process group.  The host logic of the split
(plan, strip_config) is tested beside them.
"""
import os
import socket
import sys

import numpy as np
import pytest

from oracle.oracle import from_config as oracle_from_config
from paper_2104_06784_gb300 import decomp as D
from paper_2104_06784_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class OracleStrip:
    """A strip whose engine is the FP64 oracle on the strip's window; row
    buffers are torch CPU tensors (the gloo path)."""

    def __init__(self, cfg, p):
        import torch
        self.torch = torch
        self.p = p
        self.o = oracle_from_config(D.strip_config(cfg, p))
        self.amax = None

    def get_rows(self, j0, n):
        return self.torch.from_numpy(np.ascontiguousarray(self.o.get_U()[:, j0:j0 + n]))

    def set_rows(self, j0, n, rows):
        U = self.o.get_U()
        U[:, j0:j0 + n] = rows.numpy()
        self.o.set_U(U)

    def step(self):
        self.o.step_amax(self.amax)

    def max_speed(self):
        return self.o.max_speed_rows(*self.p.own_local)

    def set_max_speed(self, v):
        self.amax = float(v)

    def own_state(self):
        a, b = self.p.own_local
        return self.o.get_U()[:, a:b]


def _spectral(nx=40, ny=66, bc=1, **over):
    rng = np.random.default_rng(7)
    dem = W.spectral_dem(nx, ny, 5.0, 2.2, 60.0, seed=4) + rng.random((ny, nx))
    h = W.parabolic_cap(nx, ny, 5.0, 5.0, nx // 2, ny // 2, 9, 3.0)
    h[ny // 5, nx // 3] += 1.0  # a second wet spot near a split
    return dict(name="spectral", dem=dem, dx=5.0, dy=5.0, params=W.default_params(bc=(bc,) * 4, cfl=0.3, **over),
                h=h, phi_s=np.full((ny, nx), 0.6),
                vx_s=np.full((ny, nx), 1.5), vy_s=np.full((ny, nx), -2.0))


def _run_decomposed(cfg, world, nsteps):
    o = D.overlap_rows(cfg["params"])
    strips = [OracleStrip(cfg, p) for p in D.plan(cfg["dem"].shape[0], world, o)]
    D.LocalComm(strips).run(nsteps)
    return np.concatenate([s.own_state() for s in strips], axis=1), strips


def test_plan_covers_every_row_once_with_overlap():
    for ny, world, o in ((66, 3, 5), (20, 4, 5), (97, 5, 7), (10, 1, 5)):
        ps = D.plan(ny, world, o)
        assert [p.own0 for p in ps][0] == 0 and ps[-1].own1 == ny
        for a, b in zip(ps, ps[1:]):
            assert a.own1 == b.own0
            assert a.win1 == a.own1 + o and b.win0 == b.own0 - o
        assert all(p.own1 - p.own0 >= (o if world > 1 else 1) for p in ps)
        assert max(p.own1 - p.own0 for p in ps) - min(p.own1 - p.own0 for p in ps) <= 1
    with pytest.raises(ValueError):
        D.plan(19, 4, 5)  # 4 rows a strip < 5 rows of overlap


def test_overlap_rows():
    assert D.overlap_rows(dict(rk=2)) == 5
    assert D.overlap_rows(dict(rk=3)) == 7


def test_strip_config_slices_and_sides():
    cfg = W.inflow_config(nx=24, ny=90, inlet_cells=6)  # west inlet, rows 42..47
    ps = D.plan(90, 3, 5)
    for p in ps:
        c = D.strip_config(cfg, p)
        assert c["dem"].shape == (p.win1 - p.win0, 24)
        assert np.array_equal(c["dem"], cfg["dem"][p.win0:p.win1])
        bc = c["params"]["bc"]
        assert bc[0] == bc[1] == 1
        assert bc[2] == (1 if p.win0 > 0 else cfg["params"]["bc"][2])
        assert bc[3] == (1 if p.win1 < 90 else cfg["params"]["bc"][3])
    c1 = D.strip_config(cfg, ps[1])  # own 30..59, window 25..64
    assert c1["inflow"]["i0"] == 42 - 25 and c1["inflow"]["i1"] == 48 - 25
    assert D.strip_config(cfg, ps[0])["inflow"] is None
    bad = dict(cfg, inflow=dict(cfg["inflow"], i0=32, i1=38))  # crosses the edge of rank 0's window (rows 0 .. 34)
    with pytest.raises(ValueError):
        D.strip_config(bad, ps[0])
    south = dict(cfg, inflow=dict(cfg["inflow"], side=2, i0=3, i1=9))
    assert D.strip_config(south, ps[0])["inflow"]["side"] == 2
    assert D.strip_config(south, ps[1])["inflow"] is None


@pytest.mark.parametrize("world", [2, 3, 4])
@pytest.mark.parametrize("bc", [0, 1])
def test_strips_equal_the_undecomposed_oracle_bit_for_bit(world, bc):
    cfg = _spectral(bc=bc)
    n = 30
    ref = oracle_from_config(cfg)
    ref.step(n)
    got, strips = _run_decomposed(cfg, world, n)
    assert np.array_equal(got, ref.get_U())
    # every strip kept the undecomposed clock
    assert all(s.o.t == ref.t for s in strips)
    # mass lies on both sides of a split (the test is not vacuous)
    U = ref.get_U()
    assert any(U[0, s.p.own1 - 1].any() and U[0, s.p.own1].any() for s in strips[:-1])


def test_three_stage_runge_kutta_and_earth_pressure():
    for over in (dict(rk=3), dict(k_mode=1)):
        cfg = _spectral(**over)
        ref = oracle_from_config(cfg)
        ref.step(20)
        got, _ = _run_decomposed(cfg, 4, 20)
        assert np.array_equal(got, ref.get_U()), over


def test_west_inflow_inside_one_window():
    cfg = W.inflow_config(nx=24, ny=90, inlet_cells=6, cfl=0.3)
    ref = oracle_from_config(cfg)
    ref.step(40)
    got, _ = _run_decomposed(cfg, 3, 40)
    assert np.count_nonzero(ref.get_U()[0]) > 0
    assert np.array_equal(got, ref.get_U())


def _dense(rk):
    """Mass and motion on every cell: every stencil reads everything it can."""
    nx, ny = 24, 66
    rng = np.random.default_rng(3)
    dem = W.spectral_dem(nx, ny, 5.0, 2.2, 60.0, seed=4) + rng.random((ny, nx))
    st = W.random_state(nx, ny, seed=5, depth=1.0, speed=1.0, dry_frac=0.0)
    return dict(name="dense", dem=dem, dx=5.0, dy=5.0, params=W.default_params(bc=(1,) * 4, cfl=0.2, rk=rk), **st)


@pytest.mark.parametrize("rk", [2, 3])
def test_the_overlap_rule_is_the_smallest_that_holds(rk):
    """On a state with mass and motion everywhere the rule's overlap gives
    the undecomposed run bit for bit, and one row less departs within ten
    steps (the own rows next to a split read a wrong value)."""
    cfg = _dense(rk)
    ref = oracle_from_config(cfg)
    ref.step(10)
    o = D.overlap_rows(cfg["params"])
    for oo, same in ((o, True), (o - 1, False)):
        strips = [OracleStrip(cfg, p) for p in D.plan(66, 4, oo)]
        D.LocalComm(strips).run(10)
        got = np.concatenate([s.own_state() for s in strips], axis=1)
        assert np.array_equal(got, ref.get_U()) == same, (rk, oo)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2104_06784_gb300 import decomp
    from tests.test_decomp_cpu import OracleStrip, _spectral
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfg = _spectral()
    p = decomp.plan(cfg["dem"].shape[0], world, decomp.overlap_rows(cfg["params"]))[rank]
    s = OracleStrip(cfg, p)
    decomp.TorchComm(s, device="cpu").run(25)
    parts = [None] * world
    dist.all_gather_object(parts, (s.own_state(), s.o.t))
    if rank == 0:
        out.put(parts)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_the_undecomposed_oracle():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    parts = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    ref = oracle_from_config(_spectral())
    ref.step(25)
    assert np.array_equal(np.concatenate([u for u, _ in parts], axis=1), ref.get_U())
    assert all(t == ref.t for _, t in parts)
