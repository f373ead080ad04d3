"""The double-float evaluation of the flux phase (moses_debug_flux_eval): the
stage's central face flux (Sect. 2.2, App. A fluxes) computed in FP64 and in
double-float arithmetic (pairs of FP32 numbers; not IEEE FP64) on synthetic
faces.  The FP64 flux is the stage kernel's own, which the stage parity tests
hold to 1e-10 of the oracle; the double-float fluxes must stay within 1e-12
of it (relative max-norm), far inside that bar, so that a double-float flux
phase would meet the FP64 form's tolerance on its own."""
import pytest

from paper_2104_06784_gb300 import moses

pytestmark = pytest.mark.gpu


def test_double_float_flux_matches_fp64():
    r = moses.flux_eval(n=1 << 20, reps=6)
    assert r["f64_gfaces_per_s"] > 0 and r["df_gfaces_per_s"] > 0
    # about 48 significant bits: a few 1e-15 relative per operation
    assert r["relmax_vs_f64"] < 1e-12, r
    # one component of one face, relative to itself: where the flux is a
    # near-cancelling sum (a flux component 1e-6 of its largest value), the
    # absolute error of the terms shows (measured 8.5e-10 on GB300)
    assert r["max_rel_vs_f64"] < 1e-8, r


def test_flux_eval_rejects_bad_sizes():
    with pytest.raises(moses.MosesError):
        moses.flux_eval(n=0, reps=6)
    with pytest.raises(moses.MosesError):
        moses.flux_eval(n=1024, reps=2)
