"""The FP64 oracle against closed forms, invariants and exact identities.

See ``tests/oracle_pins.py`` for what each pin checks and which passage of
arXiv:2104.06784 it exercises.  CPU only.
"""
import pytest

from tests import oracle_pins as P


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=[p.__name__ for p in P.ALL_PINS])
def test_pin(pin):
    pin()


def test_printed_fluid_pressure_source_breaks_the_plane_equilibrium():
    """With Eq. SrcF_f_Topo as printed (phi^f in front of grad P) a fluid-rich
    mixture in the fluid's own equilibrium on a plane does not stay at rest;
    with the reaction reading (phi^s) it does.  This documents reading R1."""
    m_printed, scale = P._plane_equilibrium(None, phi_s=0.3, delta_b=25.0, fluid_pg_mode=1)
    m_read, _ = P._plane_equilibrium(None, phi_s=0.3, delta_b=25.0, fluid_pg_mode=0)
    assert m_read < 1e-12 * scale
    assert m_printed > 1e-3 * scale
