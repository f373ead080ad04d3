"""Canary test for out-of-stencil reads (the sanitizer substitute of this
pool): the never-read pitch padding of every device plane is filled with NaN,
and runs of the stage, the ensemble and the adjoint must then give bit for bit
what the same runs give without the poison.  A kernel that read a padding
element would carry the NaN into its result."""
import numpy as np
import pytest

from paper_2104_06784_gb300 import moses, workloads as W

pytestmark = pytest.mark.gpu


def _cases():
    return [
        W.release_config(nx=77, ny=53, cfl=0.2),                       # closed boundaries
        W.inflow_config(nx=61, ny=40, dx=5.0, inlet_cells=6),          # inflow ghosts
        W.large_release_config(n=70, ny=45, dx=10.0, seed=3, volume=1e5, radius_cells=6),  # transmissive
        W.release_config(nx=45, ny=30, cfl=0.2, nu_f=1.0),             # viscous form (3 x 3 stencil)
    ]


@pytest.mark.parametrize("precision", [moses.FP64, moses.FP32])
@pytest.mark.parametrize("case", range(4))
def test_steps_ignore_padding(precision, case):
    cfg = _cases()[case]
    a = moses.from_config(cfg, precision=precision)
    b = moses.from_config(cfg, precision=precision)
    b.debug_poison()
    for tile in (0, 1, 2, 3):
        a.set_tile(tile)
        b.set_tile(tile)
        a.step(15)
        b.step(15)
    Ua, Ub = a.get_conserved(), b.get_conserved()
    assert np.isfinite(Ub).all()
    assert np.array_equal(Ua, Ub)
    assert a.budget()["t"] == b.budget()["t"]
    assert np.array_equal(a.stage(a.budget()["t"], 0.01), b.stage(b.budget()["t"], 0.01))


@pytest.mark.parametrize("precision", [moses.FP64, moses.FP32])
def test_adjoint_ignores_padding(precision):
    cfg = W.large_release_config(n=70, ny=45, dx=10.0, seed=3, volume=1e5, radius_cells=6)
    target = np.zeros((45, 70))
    ra = moses.from_config(cfg, precision=precision).adjoint_misfit(30, target, ckpt_every=7)
    b = moses.from_config(cfg, precision=precision)
    b.debug_poison()
    rb = b.adjoint_misfit(30, target, ckpt_every=7)
    assert np.isfinite(rb["g_release_h"]).all()
    assert abs(ra["loss"] - rb["loss"]) <= 1e-14 * ra["loss"]
    assert np.allclose(ra["g_params"], rb["g_params"], rtol=1e-12, atol=0)
    assert np.allclose(ra["g_release_h"], rb["g_release_h"], rtol=1e-12, atol=1e-300)


def test_batch_ignores_padding():
    cfgs = _cases()[:3]
    clean = [moses.from_config(c, precision=moses.FP32) for c in cfgs]
    poisoned = [moses.from_config(c, precision=moses.FP32) for c in cfgs]
    for s in poisoned:
        s.debug_poison()
    for group in (clean, poisoned):
        with moses.Batch(group) as bt:
            bt.step(20)
    for x, y in zip(clean, poisoned):
        assert np.array_equal(x.get_conserved(), y.get_conserved())


# ----------------------------------------------------------------------------
# failure detection: a fault injected on the host (a prescribed time step far
# beyond the CFL limit) overflows in the kernels; the device status word turns
# it into MOSES_ENONFINITE at the C-ABI instead of a silent NaN field


@pytest.mark.parametrize("precision", [moses.FP64, moses.FP32])
def test_overflow_is_reported_as_nonfinite(precision):
    cfg = W.release_config(nx=40, ny=30, cfl=0.2)
    s = moses.from_config(cfg, precision=precision)
    U0 = s.get_conserved()
    with pytest.raises(moses.MosesError) as e:
        s.step_dt(1e300 if precision == moses.FP64 else 1e30, 3)
    assert e.value.code == moses.MOSES_ENONFINITE
    with pytest.raises(moses.MosesError):  # reported again until a new state is set
        s.step(1)
    s.set_conserved(U0)
    s.step(2)
    assert np.isfinite(s.get_conserved()).all()


# ----------------------------------------------------------------------------
# the one device-side wait (the classification's wait for its bulk copies on
# an mbarrier) is bounded: made to run out -- the barrier expects bytes no
# copy delivers -- it ends, the step reports MOSES_ETIMEOUT and the context
# stays usable


@pytest.mark.parametrize("precision", [moses.FP64, moses.FP32])
def test_copy_wait_timeout_is_reported(precision):
    cfg = W.release_config(nx=40, ny=30, cfl=0.2)
    s = moses.from_config(cfg, precision=precision)
    U0 = s.get_conserved()
    s.debug_timeout(True)
    with pytest.raises(moses.MosesError) as e:
        s.step(1)
    assert e.value.code == moses.MOSES_ETIMEOUT
    s.debug_timeout(False)
    s.set_conserved(U0)  # a new state clears the status word
    s.step(5)
    ref = moses.from_config(cfg, precision=precision)
    ref.step(5)
    assert np.array_equal(s.get_conserved(), ref.get_conserved())
