"""Simulations that share one stream.  The stepping launches follow one
another as programmatic dependent launches: each kernel may start while the
kernel before it in the stream finishes, and waits before its first read of
that kernel's results.  With two simulations stepping in turn on one stream,
a simulation's kernel follows the other simulation's; each must still end
bit for bit where it ends alone (FP64 and FP32, the masked plain form and
the three-stage form)."""
import numpy as np
import pytest

from paper_2104_06784_gb300 import moses, workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [moses.FP64, moses.FP32])
@pytest.mark.parametrize("rk", [2, 3])
def test_two_simulations_in_turn_on_one_stream(precision, rk):
    torch = pytest.importorskip("torch")
    cfg_a = W.release_config(rk=rk)
    cfg_b = W.large_release_config(n=160, ny=96, dx=10.0, seed=5, volume=3e5, radius_cells=10, rk=rk)
    solo = []
    for cfg in (cfg_a, cfg_b):
        with moses.from_config(cfg, precision=precision) as s:
            s.step(60)
            solo.append(s.get_conserved())
    stream = torch.cuda.Stream()
    a = moses.from_config(cfg_a, precision=precision, stream=stream)
    b = moses.from_config(cfg_b, precision=precision, stream=stream)
    try:
        b.set_tile(3)  # the two-thread tile form beside the default one
        for _ in range(20):
            a.step(3)
            b.step(3)
        assert np.array_equal(a.get_conserved(), solo[0])
        assert np.array_equal(b.get_conserved(), solo[1])
    finally:
        a.close()
        b.close()
