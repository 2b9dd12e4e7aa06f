"""Pins of the oracle's diagnostics (Section 6.1: the bubble's centroid and rise
velocity; the phase mass and momentum) against symmetry, closed forms and
special cases -- none of them re-types the definitions."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as orc
import workloads as W


def _bubble(nx, ny, nz, centre, radius, xi=5.0, walls=(1, 1, 1)):
    prob = W.Problem(nx, ny, nz, wall=walls, xi=xi, clamp_phi=1)
    return prob, W.sphere_phi(prob, centre, radius, heavy_inside=False)


def test_centroid_of_a_symmetric_bubble_is_its_centre():
    # the cell centres i + 1/2 are symmetric about any integer point, so the
    # indicator-weighted centroid is the sphere's centre; distinct coordinates
    # per axis catch a transposed axis, the + 1/2 catches an index offset
    prob, phi = _bubble(26, 34, 22, (11.0, 19.0, 10.0), 6.0)
    d = orc.diagnostics(prob, phi, np.zeros((3,) + prob.shape))
    assert d["light_x"] == pytest.approx(11.0, abs=1e-12)
    assert d["light_y"] == pytest.approx(19.0, abs=1e-12)
    assert d["light_z"] == pytest.approx(10.0, abs=1e-12)
    assert d["light_ux"] == d["light_uy"] == d["light_uz"] == 0.0 and d["max_u"] == 0.0


def test_light_volume_is_the_integral_of_the_indicator():
    # b = clamp(1 - 2 phi, 0, 1) = tanh(2 (R - r) / xi) inside r < R and 0 outside
    # for the light-inside tanh profile: the cell sum approximates the radial
    # integral 4 pi int_0^R r^2 tanh(2 (R - r) / xi) dr (a 1 - phi weight would
    # add the heavy-side tail and overshoot by tens of percent)
    R, xi = 10.0, 5.0
    prob, phi = _bubble(40, 40, 40, (20.0, 20.0, 20.0), R, xi)
    exact = integrate.quad(lambda r: 4 * math.pi * r * r * math.tanh(2 * (R - r) / xi), 0.0, R)[0]
    d = orc.diagnostics(prob, phi, np.zeros((3,) + prob.shape))
    assert d["light_vol"] == pytest.approx(exact, rel=5e-3)
    assert (1.0 - phi).sum() > 1.2 * exact


def test_uniform_velocity_and_momentum():
    prob, phi = _bubble(20, 28, 18, (10.0, 12.0, 9.0), 5.0)
    vel = np.array([1e-3, -2.5e-3, 4e-4])
    u = np.broadcast_to(vel[:, None, None, None], (3,) + prob.shape).copy()
    d = orc.diagnostics(prob, phi, u)
    rho = prob.rho_L + np.clip(phi.astype(np.float64), 0, 1) * (prob.rho_H - prob.rho_L)
    total_mass = rho.sum()
    for a, name in enumerate("xyz"):
        assert d["light_u" + name] == pytest.approx(vel[a], rel=1e-12)
        assert d["mom_" + name] == pytest.approx(vel[a] * total_mass, rel=1e-12)
    assert d["max_u"] == pytest.approx(np.linalg.norm(vel), rel=1e-12)
    assert d["mass"] == pytest.approx(phi.astype(np.float64).sum(), rel=1e-14)


def test_velocity_equal_to_position_gives_the_centroid():
    # u_a = a + 1/2 at every cell: the bubble's mean velocity equals its centroid
    prob, phi = _bubble(24, 30, 20, (9.3, 17.7, 11.1), 5.5)
    z, y, x = np.meshgrid(np.arange(20) + .5, np.arange(30) + .5, np.arange(24) + .5, indexing="ij")
    d = orc.diagnostics(prob, phi, np.stack([x, y, z]))
    for name in "xyz":
        assert d["light_u" + name] == pytest.approx(d["light_" + name], rel=1e-12)
    # an off-grid centre: the centroid sits within a fraction of a cell of it
    assert d["light_x"] == pytest.approx(9.3, abs=0.05) and d["light_y"] == pytest.approx(17.7, abs=0.05)


@pytest.mark.parametrize("clamp", [0, 1])
def test_density_clamp_in_the_momentum(clamp):
    # phi below 0 (the undershoot at high density ratio): with the clamp the
    # density is rho_L there, without it rho_L + phi (rho_H - rho_L) < rho_L
    prob = W.Problem(6, 5, 4, rho_ratio=1000.0, clamp_phi=clamp)
    phi = np.full(prob.shape, -4e-4)
    u = np.zeros((3,) + prob.shape)
    u[1] = 2.0
    d = orc.diagnostics(prob, phi, u)
    rho = prob.rho_L if clamp else prob.rho_L - 4e-4 * (prob.rho_H - prob.rho_L)
    assert d["mom_y"] == pytest.approx(2.0 * rho * prob.ncells, rel=1e-12)
    assert d["light_vol"] == pytest.approx(prob.ncells, rel=1e-15)  # b = clamp(1.0008) = 1


def test_heavy_bulk_does_not_enter_the_bubble():
    # phi >= 1/2 everywhere (a heavy box with acoustic ripples): no light volume
    prob = W.Problem(8, 8, 8)
    rng = np.random.default_rng(0)
    phi = 1.0 + 1e-4 * rng.standard_normal(prob.shape)
    d = orc.diagnostics(prob, phi, np.zeros((3,) + prob.shape))
    assert d["light_vol"] == 0.0 and d["light_y"] == 0.0
