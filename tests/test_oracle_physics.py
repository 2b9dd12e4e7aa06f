"""Physics pins of the FP64 oracle: closed forms of the continuum equations that
the scheme of Section 3 must reproduce on small boxes.

* phase-field diffusion: with theta -> 0 (xi -> infinity), no flow, the phase
  LB solves d(phi)/dt = M lap(phi), so a sine mode decays at M k^2
  (eq:allen_cahn, eq:mobility: pins omega_phi = 1/(3M + 1/2));
* shear wave: a uniform-phi shear wave decays at nu k^2 with
  nu = tau c_s^2, tau = tau_L + phi (tau_H - tau_L), s_nu = 1/(tau + 1/2);
* planar interface: the tanh profile of Section 3.1 is (close to) steady;
* advection: a uniform flow carries the interface at its speed;
* Laplace law: the pressure jump across a circular / spherical interface is
  sigma/R (2-D) and 2 sigma/R (3-D), given beta = 12 sigma/xi,
  kappa = 3 sigma xi/2 (eq:chemPot);
* two-layer Poiseuille: the sharp-interface textbook profile and the exact
  solution of d/dy(mu(y) du/dy) = -rho(y) G for the diffuse profile (this
  needs the viscous force F_mu of eq:viscousForce when rho varies);
* hydrostatics: p(bottom) - p(top) equals the integral of rho g (this needs
  the pressure force F_p = -p* c_s^2 grad(rho) of eq:pressure_force).
"""
import numpy as np
import pytest
from scipy.integrate import cumulative_trapezoid

import workloads as W

CS2 = 1.0 / 3.0


def _equilibrium_flow(orc, s, prob, u):
    """Sets g = g^eq(p* = 0, u) and h = phi Gamma(u) (state construction only)."""
    e, w, _ = orc.lattice(prob.q_hydro)
    eh, wh, _ = orc.lattice(prob.q_phase)
    uu = (u ** 2).sum(0)
    eu = np.einsum("ia,a...->i...", e.astype(float), u)
    s.g[:] = w[:, None, None, None] * (3 * eu + 4.5 * eu ** 2 - 1.5 * uu)
    ehu = np.einsum("ia,a...->i...", eh.astype(float), u)
    s.h[:] = wh[:, None, None, None] * (1 + 3 * ehu + 4.5 * ehu ** 2 - 1.5 * uu) * s.phi_prev[None]
    s.u_prev[:] = u


@pytest.mark.parametrize("mrt,qp", [(0, 15), (1, 15), (0, 27), (1, 19)])
def test_phase_diffusion_rate(orc, mrt, qp):
    """A sine mode of phi decays at M k^2 (eq:mobility, reading A2).  The
    diffusivity is set by the relaxation of the first-order moments alone, so the
    MRT phase collision (Section 3.1: other moments relaxed with 1) decays at the
    same rate."""
    prob = W.Problem(64, 1, 1, q_hydro=19, rho_ratio=1.0, mu_ratio=1.0, nu_H=0.1, sigma=0.0, xi=1e9,
                     mobility=0.05, phase_mrt=mrt, q_phase=qp)
    p = orc.make_problem(prob)
    x = np.arange(64) + 0.5
    k = 2 * np.pi / 64
    s = orc.State(p, (0.5 + 0.1 * np.sin(k * x)).reshape(1, 1, 64))
    amps = []
    for T in (500, 2500):
        s.run(T - s.k)
        amps.append(np.sum((s.phi()[0, 0] - 0.5) * np.sin(k * x)))
    rate = np.log(amps[0] / amps[1]) / 2000
    assert rate == pytest.approx(prob.mobility * k * k, rel=5e-3)


@pytest.mark.parametrize("q", [19, 27])
def test_shear_wave_viscosity(orc, q):
    phi_u = 0.3
    prob = W.Problem(1, 64, 1, q_hydro=q)
    p = orc.make_problem(prob)
    y = np.arange(64) + 0.5
    k = 2 * np.pi / 64
    s = orc.State(p, np.full((1, 64, 1), phi_u))
    u = np.zeros((3, 1, 64, 1))
    u[0, 0, :, 0] = 1e-3 * np.sin(k * y)
    _equilibrium_flow(orc, s, prob, u)
    amps = []
    for T in (200, 2200):
        s.run(T - s.k)
        _, uf, _ = s.fields()
        amps.append(np.sum(uf[0, 0, :, 0] * np.sin(k * y)))
    rate = np.log(amps[0] / amps[1]) / 2000
    tau = 3 * prob.nu_L + phi_u * (3 * prob.nu_H - 3 * prob.nu_L)
    assert rate == pytest.approx(tau * CS2 * k * k, rel=5e-3)


@pytest.mark.parametrize("q,qp", [(19, 15), (27, 15), (19, 19), (27, 27)])
def test_planar_interface_steady(orc, q, qp):
    prob = W.Problem(64, 1, 1, q_hydro=q, q_phase=qp)  # rho ratio 1000, sigma 1e-4, xi 5, M 0.02
    p = orc.make_problem(prob)
    phi0 = W.slab_phi(prob, 16.0, 48.0)
    s = orc.State(p, phi0)
    m0 = s.phi().sum()
    s.run(2000)
    phi, u, _ = s.fields()
    assert np.abs(phi - phi0).max() < 1e-2
    assert np.abs(u).max() < 1e-6
    assert abs(phi.sum() - m0) < 1e-12 * m0


def test_interface_advection(orc):
    prob = W.Problem(64, 1, 1, q_hydro=19, rho_ratio=1.0, mu_ratio=1.0, nu_H=0.05, sigma=0.0)
    p = orc.make_problem(prob)
    s = orc.State(p, W.slab_phi(prob, 16.0, 40.0))
    U = np.zeros((3, 1, 1, 64))
    U[0] = 0.02
    _equilibrium_flow(orc, s, prob, U)
    s.run(800)  # shift 0.02 * 800 = 16 cells
    assert np.abs(s.phi() - W.slab_phi(prob, 32.0, 56.0)).max() < 1.5e-2


def _laplace_cylinder(orc, R, n=48, steps=3000, sigma=1e-3, q=19, qp=15):
    prob = W.Problem(n, n, 1, q_hydro=q, q_phase=qp, rho_ratio=1.0, mu_ratio=1.0, nu_H=0.1, sigma=sigma, xi=4.0,
                     mobility=0.05)
    s = orc.State(orc.make_problem(prob), W.cylinder_phi(prob, (n / 2, n / 2), R, heavy_inside=True))
    s.run(steps)
    phi, u, pr = s.fields()
    R_eff = np.sqrt(phi.sum() / np.pi)
    return R_eff, pr[0, n // 2, n // 2] - pr[0, 0, 0], np.abs(u).max()


def test_laplace_law_cylinder(orc):
    sigma = 1e-3
    pts = [_laplace_cylinder(orc, R, sigma=sigma) for R in (8.0, 11.0, 14.0)]
    inv_r = np.array([1 / r for r, _, _ in pts])
    dp = np.array([d for _, d, _ in pts])
    slope = np.polyfit(inv_r, dp, 1)[0]
    assert slope == pytest.approx(sigma, rel=5e-2)
    assert all(umax < 1e-5 for _, _, umax in pts)


def test_laplace_law_sphere(orc):
    n, R, sigma = 24, 6.0, 1e-3
    prob = W.Problem(n, n, n, q_hydro=19, rho_ratio=1.0, mu_ratio=1.0, nu_H=0.1, sigma=sigma, xi=4.0,
                     mobility=0.05)
    s = orc.State(orc.make_problem(prob), W.sphere_phi(prob, (n / 2,) * 3, R, heavy_inside=True))
    s.run(1500)
    phi, u, pr = s.fields()
    R_eff = (3 * phi.sum() / (4 * np.pi)) ** (1 / 3)
    dp = pr[n // 2, n // 2, n // 2] - pr[0, 0, 0]
    assert dp == pytest.approx(2 * sigma / R_eff, rel=1e-1)


def _two_layer(orc, ratio, mu_ratio, nu_H, xi, q=19, H=64, G=1e-6, steps=40000):
    """Channel between walls at y = 0 and y = H (half-way bounce-back), heavy fluid
    on top, light below, driven by F_b = rho G x (rho_ref = 0)."""
    prob = W.Problem(1, H, 1, wall=(0, 1, 0), q_hydro=q, rho_ratio=ratio, mu_ratio=mu_ratio, nu_H=nu_H,
                     sigma=1e-4, xi=xi, mobility=0.05, gravity=(G, 0, 0), rho_ref=0.0)
    y = np.arange(H) + 0.5
    phi0 = (0.5 + 0.5 * np.tanh(2 * (y - H / 2) / xi)).reshape(1, H, 1)
    s = orc.State(orc.make_problem(prob), phi0)
    s.run(steps)
    _, u, _ = s.fields()
    return prob, y, u[0, 0, :, 0]


def _diffuse_exact(prob, G, H, y):
    """u(y) solving d/dy(mu du/dy) = -rho G, u(0) = u(H) = 0, with rho, nu linear
    in the tanh profile phi(y) (fine quadrature)."""
    yf = np.linspace(0, H, 200 * H + 1)
    phi = 0.5 + 0.5 * np.tanh(2 * (yf - H / 2) / prob.xi)
    rho = prob.rho_L + phi * (prob.rho_H - prob.rho_L)
    mu = rho * (prob.nu_L + phi * (prob.nu_H - prob.nu_L))
    S = cumulative_trapezoid(rho * G, yf, initial=0)
    I1 = cumulative_trapezoid(1 / mu, yf, initial=0)
    I2 = cumulative_trapezoid(S / mu, yf, initial=0)
    return np.interp(y, yf, I2[-1] / I1[-1] * I1 - I2)


def _l2(a, b):
    return np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum())


def test_two_layer_poiseuille_sharp(orc):
    """Textbook sharp-interface solution; the diffuse interface (xi/h = 1/8) with
    a 10x viscosity contrast keeps it within 10 %."""
    G, H = 1e-6, 64
    prob, y, ux = _two_layer(orc, 1.0, 10.0, nu_H=0.5, xi=4.0, steps=30000)
    h, yy = H / 2, y - H / 2
    mu1, mu2 = prob.rho_H * prob.nu_H, prob.rho_L * prob.nu_L
    f1, f2 = prob.rho_H * G, prob.rho_L * G
    a1 = h * (f1 / mu1 - f2 / mu2) * mu2 / (2 * (mu1 + mu2))
    a2 = mu1 * a1 / mu2
    b = f1 * h * h / (2 * mu1) - a1 * h
    ua = np.where(yy > 0, -f1 * yy ** 2 / (2 * mu1) + a1 * yy + b, -f2 * yy ** 2 / (2 * mu2) + a2 * yy + b)
    assert _l2(ux, ua) < 0.10


@pytest.mark.parametrize("ratio,mu_ratio,nu_H,xi,q,tol", [
    (1.0, 10.0, 0.5, 4.0, 19, 2e-3),
    (10.0, 1.0, 0.05, 8.0, 19, 1.5e-2),
    (1000.0, 100.0, 0.05, 4.0, 27, 1e-2),
])
def test_two_layer_poiseuille_diffuse(orc, ratio, mu_ratio, nu_H, xi, q, tol):
    prob, y, ux = _two_layer(orc, ratio, mu_ratio, nu_H=nu_H, xi=xi, q=q)
    assert _l2(ux, _diffuse_exact(prob, 1e-6, 64, y)) < tol


@pytest.mark.parametrize("ratio", [10.0, 1000.0])
def test_hydrostatic_balance(orc, ratio):
    H, g = 64, 1e-5
    prob = W.Problem(1, H, 1, wall=(0, 1, 0), q_hydro=19, rho_ratio=ratio, mu_ratio=100.0, nu_H=0.1,
                     sigma=1e-4, xi=4.0, mobility=0.05, gravity=(0, -g, 0), rho_ref=0.0)
    y = np.arange(H) + 0.5
    phi0 = (0.5 - 0.5 * np.tanh(2 * (y - H / 2) / prob.xi)).reshape(1, H, 1)  # heavy below
    s = orc.State(orc.make_problem(prob), phi0)
    s.run(20000)
    phi, u, pr = s.fields()
    P = pr[0, :, 0]
    rho = prob.rho_L + phi[0, :, 0] * (prob.rho_H - prob.rho_L)
    exact = g * np.sum(0.5 * (rho[2:-3] + rho[3:-2]))
    assert P[2] - P[-3] == pytest.approx(exact, rel=1.5e-2)
    assert np.abs(u).max() < 2e-5
