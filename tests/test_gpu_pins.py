"""The GPU path (FP64 form, through the C-ABI) against the same analytic pins
as the oracle: closed-box conservation, bodies at rest (lake, mixture, heap),
the Ritter dam break, the Savage-Hutter similarity solution, drag and wave
speeds, 90-degree rotation invariance, the closed box, the viscous and fluid
friction checks, the central-upwind pins, the WENO / three-stage
Runge-Kutta pins and the earth-pressure pins (regimes, similarity solutions
spreading and contracting, celerity, rotation).  Each pin builds its inputs and
runs a simulation through `_sim`; here `_sim` returns a GPU simulation with
the oracle's interface, so the kernels are checked against closed forms and
invariants directly, not only against the oracle.  (Pins that read the
oracle's geometry arrays or its inflow ghost state have no GPU counterpart.)
"""
import numpy as np
import pytest

from tests import oracle_pins as P
from paper_2104_06784_gb300 import moses

pytestmark = pytest.mark.gpu


class GpuSim:
    """moses.Sim behind the interface of oracle.OracleSim used by the pins."""

    def __init__(self, dem, dx, dy, params, precision=moses.FP64):
        self.params = dict(params)
        self.s = moses.Sim(np.asarray(dem, dtype=np.float64), dx, dy, self.params, precision=precision)
        self.ny, self.nx = self.s.ny, self.s.nx

    def set_release(self, h, phi_s, vx_s=None, vy_s=None, vx_f=None, vy_f=None):
        self.s.set_release(h, phi_s, vx_s, vy_s, vx_f, vy_f)

    def set_inflow(self, side, i0, i1, t, Q, phi):
        self.s.set_inflow(side, i0, i1, t, Q, phi)

    def set_U(self, U):
        self.s.set_conserved(U)

    def get_U(self):
        return self.s.get_conserved()

    def step(self, n=1):
        self.s.step(n)

    def step_dt(self, dt):
        self.s.step_dt(dt, 1)

    def stage(self, t, dt):
        return self.s.stage(t, dt)

    def cfl_dt(self):
        return self.s.next_dt()[0]

    def max_speed(self):
        return self.s.max_speed()

    def budget(self):
        return self.s.budget()

    def primitive(self):
        return self.s.get_state()

    @property
    def t(self):
        return self.s.budget()["t"]


GPU_PINS = [P.pin_conservation_closed, P.pin_lake_flat, P.pin_lake_plane, P.pin_mixture_plane_rest,
            P.pin_mixture_no_separation, P.pin_heap_rest, P.pin_ritter, P.pin_savage_hutter, P.pin_drag,
            P.pin_wave_speed, P.pin_rotation, P.pin_friction, P.pin_closed_box, P.pin_viscous,
            P.pin_fluid_friction, P.pin_cu_upwind_dependence, P.pin_cu_conservation_and_ritter, P.pin_cu_rotation,
            P.pin_weno_linear_exact, P.pin_weno_rk3_dam_break, P.pin_weno_smooth_order, P.pin_rk3_drag_factor,
            P.pin_weno_rk3_budgets_and_rotation,
            P.pin_lake_curved_bed_residual_converges,
            P.pin_earth_pressure_regimes, P.pin_earth_pressure_fluid_unaffected, P.pin_earth_pressure_wave_speed,
            P.pin_savage_hutter_earth_pressure, P.pin_rotation_earth_pressure]


@pytest.mark.parametrize("pin", GPU_PINS, ids=lambda f: f.__name__)
def test_gpu_satisfies_pin(pin, monkeypatch):
    monkeypatch.setattr(P, "_sim", lambda dem, dx, dy, params, L: GpuSim(dem, dx, dy, params))
    pin()
