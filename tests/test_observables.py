"""Host arithmetic of the rising-bubble observables (Section 6.1), against closed
forms and a synthetic record."""
import math

import numpy as np
import pytest

import workloads as W
from paper_2012_06144_gb300 import observables as O


def test_drag_correlation_limits():
    # large Re: the spherical-cap constant 2.67; small Re: Stokes-like 16 / Re
    assert O.drag_correlation(1e12) == pytest.approx(2.67, rel=1e-9)
    for re in (1e-4, 1e-3):  # [b^0.9 + a^0.9]^(10/9) = b (1 + (10/9)(a/b)^0.9 + ...), a/b = 2.67 Re / 16
        assert O.drag_correlation(re) == pytest.approx(16.0 / re, rel=1.2 * (10 / 9) * (2.67 * re / 16.0) ** 0.9)
    # where the two terms are equal the sum doubles inside the bracket
    assert O.drag_correlation(16.0 / 2.67) == pytest.approx(2.0 ** (10.0 / 9.0) * 2.67, rel=1e-12)
    re = np.logspace(-1, 3, 50)
    cd = np.array([O.drag_correlation(r) for r in re])
    assert np.all(np.diff(cd) < 0)


def test_drag_coefficient_balances_buoyancy():
    g, rho_H, rho_L, D = 8e-6, 1.0, 1e-3, 32.0
    for cd in (0.5, 1.0, 2.67, 10.0):
        # drag cd rho_H u^2 / 2 * pi D^2 / 4 equals buoyancy (rho_H - rho_L) g pi D^3 / 6
        u = math.sqrt(4.0 / 3.0 * g * (rho_H - rho_L) * D / (rho_H * cd))
        assert O.drag_coefficient(g, rho_H, rho_L, D, u) == pytest.approx(cd, rel=1e-12)
        drag = cd * rho_H * u * u / 2 * math.pi * D * D / 4
        assert drag == pytest.approx((rho_H - rho_L) * g * math.pi * D ** 3 / 6, rel=1e-12)


def test_groups_match_the_rising_bubble_recipe():
    prob, _ = W.rising_bubble()  # Eo 10, Mo 1e-3, t_ref 2000, D 32
    g = -prob.gravity[1]
    assert O.eotvos(prob.rho_H, g, 32.0, prob.sigma) == pytest.approx(10.0, rel=1e-12)
    assert O.gravity_reynolds(prob.rho_H, g, 32.0, prob.rho_H * prob.nu_H) == pytest.approx(1e6 ** 0.25, rel=1e-12)
    assert O.reference_time(32.0, g) == pytest.approx(2000.0, rel=1e-12)


class _FakeRise:
    """A bubble that accelerates to u_t with time constant tau, as seen by
    lbm_reduce."""

    def __init__(self, u_t=0.01, tau=300.0, y0=64.0):
        self.t, self.u_t, self.tau, self.y0 = 0, u_t, tau, y0

    def step(self, n):
        self.t += n

    def steps_done(self):
        return self.t

    def reduce(self):
        t, tau = self.t, self.tau
        y = self.y0 + self.u_t * (t - tau * (1.0 - math.exp(-t / tau)))
        return dict(light_x=64.0, light_y=y, light_z=64.0, light_ux=0.0, light_uy=self.u_t * (1.0 - math.exp(-t / tau)),
                    light_uz=0.0, light_vol=4000.0, max_u=2 * self.u_t)


def test_track_and_summary_on_a_known_rise():
    prob, _ = W.rising_bubble()
    rec = O.track(_FakeRise(), steps=10000, every=100)
    t, c, v, vol, _ = rec.arrays()
    assert t[0] == 0 and t[-1] == 10000 and len(t) == 101
    u_t, spread = O.terminal_velocity(rec, t_ref=2000.0, window=1.0)
    assert u_t == pytest.approx(0.01, rel=1e-3) and spread < 1e-2
    assert O.mean_core_velocity(rec, 2000.0, 1.0) == pytest.approx(0.01, rel=1e-3)
    dv = O.centroid_velocity(rec)[5:-1]
    assert np.allclose(dv, v[5:-1, 1], rtol=2e-2)
    s = O.summary(prob, rec, 32.0, window=1.0)
    assert s["C_D"] == pytest.approx(O.drag_coefficient(8e-6, 1.0, 1e-3, 32.0, u_t), rel=1e-12)
    assert s["Re_t"] == pytest.approx(u_t * 32.0 / prob.nu_H, rel=1e-12)
    assert s["t_star_end"] == pytest.approx(5.0) and s["light_volume_drift"] == 0.0
