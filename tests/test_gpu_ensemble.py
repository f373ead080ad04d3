"""Ensembles (moses_batch_*): members of different sizes, DEMs and parameters
advanced together, all the steps of a call in one cooperative launch whose
CTAs meet on a bounded grid barrier between the phases of a stage.

Each member must equal its solo run bit for bit (the launch runs the same tile
code) for every tile shape the tuner can choose, keep its own time and CFL
time step, and match the FP64 oracle at the parity tolerance.  A barrier
whose waits run out (moses_batch_debug_timeout: it waits for one CTA more than
the grid holds) ends the launch with MOSES_ETIMEOUT, no fault, and the batch
steps normally afterwards.
"""
import numpy as np
import pytest

from oracle.oracle import from_config as oracle_from_config
from paper_2104_06784_gb300 import moses, workloads as W

pytestmark = pytest.mark.gpu


def _members():
    cfgs = [
        W.release_config(nx=40, ny=40, cfl=0.2),
        W.release_config(nx=77, ny=53, cfl=0.1, delta_b_deg=20.0, c_d=5e-3),
        W.large_release_config(n=96, ny=72, dx=10.0, seed=4, volume=2e5, radius_cells=8),
        W.inflow_config(nx=64, ny=33, dx=5.0, inlet_cells=6),
        W.release_config(nx=33, ny=9, cfl=0.3),
    ]
    return cfgs


@pytest.mark.parametrize("rows", [None, 4, 8, 16])
@pytest.mark.parametrize("precision", [moses.FP64, moses.FP32])
def test_batch_equals_solo_runs(precision, rows):
    cfgs = _members()
    steps = 37  # two calls: 20 steps and 17 steps
    members = [moses.from_config(c, precision=precision) for c in cfgs]
    with moses.Batch(members) as b:
        ty, ms = b.tile_rows()
        assert ty in (4, 8, 16) and all(m > 0 for m in ms)
        if rows is not None:
            b.set_tile_rows(rows)
            ty = rows
        assert b.tile_rows()[0] == ty
        assert b.tiles == sum(((m.nx + 31) // 32) * ((m.ny + ty - 1) // ty) for m in members)
        b.step(20)
        b.step(steps - 20)
    times = []
    for c, m in zip(cfgs, members):
        solo = moses.from_config(c, precision=precision)
        t = solo.step(steps)
        assert np.array_equal(m.get_conserved(), solo.get_conserved()), c["name"]
        bm, bs = m.budget(), solo.budget()
        assert bm["t"] == t and bm["steps"] == steps
        assert abs(bm["vol_s"] - bs["vol_s"]) <= 1e-12 * max(bs["vol_s"], 1e-30)
        times.append(t)
    assert len(set(times)) == len(times), "members must keep their own time"


def test_batch_member_matches_oracle():
    cfgs = _members()
    members = [moses.from_config(c) for c in cfgs]
    with moses.Batch(members) as b:
        b.step(20)
    for c, m in zip(cfgs, members):
        o = oracle_from_config(c)
        o.step(20)
        Uo = o.get_U()
        scale = np.abs(Uo).reshape(6, -1).max(axis=1)
        scale = np.where(scale > 0, scale, 1.0)
        err = (np.abs(m.get_conserved() - Uo).reshape(6, -1).max(axis=1) / scale).max()
        assert err < 1e-10, (c["name"], err)


def test_batch_rejects_bad_members():
    a = moses.from_config(W.release_config(nx=20, ny=20))
    f = moses.from_config(W.release_config(nx=20, ny=20), precision=moses.FP32)
    with pytest.raises(moses.MosesError):
        moses.Batch([a, f])
    with pytest.raises(moses.MosesError):
        moses.Batch([a, a])


@pytest.mark.parametrize("precision", [moses.FP64, moses.FP32])
def test_barrier_timeout_is_reported_and_the_batch_recovers(precision):
    cfgs = _members()[:3]
    members = [moses.from_config(c, precision=precision) for c in cfgs]
    U0 = [m.get_conserved() for m in members]
    with moses.Batch(members) as b:
        b.debug_timeout(True)
        with pytest.raises(moses.MosesError) as e:
            b.step(3)
        assert e.value.code == moses.MOSES_ETIMEOUT
        # the launch ended at its first meeting: no stage reached the states
        for m, u in zip(members, U0):
            assert np.array_equal(m.get_conserved(), u)
        b.debug_timeout(False)
        b.step(12)
    for c, m in zip(cfgs, members):
        solo = moses.from_config(c, precision=precision)
        solo.step(12)
        assert np.array_equal(m.get_conserved(), solo.get_conserved()), c["name"]


def test_batch_rejects_bad_tile_rows():
    members = [moses.from_config(c) for c in _members()[:2]]
    with moses.Batch(members) as b:
        with pytest.raises(moses.MosesError):
            b.set_tile_rows(6)
