"""The two-dimensional pair of Section 5.1 -- D2Q9 for the phase field and the
hydrodynamics, on an nx x ny x 1 box -- in the FP64 oracle: lattice identities in
the plane, stencils exact on quadratics, collision moments with two-dimensional
Hermite tensors, conservation, and the two-dimensional physics pins (diffusion
rate, shear-wave viscosity, planar interface, Laplace law of a cylinder).  The
literal moment-space whole step covers D2Q9 in test_oracle_bruteforce."""
import numpy as np
import pytest

import test_oracle_identities as I
import test_oracle_physics as Ph
import workloads as W

CS2 = 1.0 / 3.0
D2 = np.diag([1.0, 1.0, 0.0])  # the identity of the plane


def test_d2q9_lattice_moments(orc):
    e, w, opp = orc.lattice(9)
    assert len(w) == 9 and len({tuple(v) for v in e}) == 9 and (e[:, 2] == 0).all()
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs(w @ e).max() < 1e-15
    assert np.abs(np.einsum("i,ia,ib->ab", w, e, e) - CS2 * D2).max() < 1e-15
    assert np.abs(np.einsum("i,ia,ib,ic->abc", w, e, e, e)).max() < 1e-15
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, e, e, e, e)
    iso = CS2 ** 2 * (np.einsum("ab,cd->abcd", D2, D2) + np.einsum("ac,bd->abcd", D2, D2)
                      + np.einsum("ad,bc->abcd", D2, D2))
    assert np.abs(m4 - iso).max() < 1e-15
    assert (e[opp] == -e).all() and (e[0] == 0).all()
    for i in range(1, 9, 2):
        assert opp[i] == i + 1


def test_d2q9_stencils_exact_on_quadratics(orc):
    rng = np.random.default_rng(21)
    prob = W.Problem(12, 10, 1, q_hydro=9, q_phase=9)
    p = orc.make_problem(prob)
    z, y, x = np.meshgrid(np.arange(1.0), np.arange(10.0), np.arange(12.0), indexing="ij")
    a = rng.normal(size=2)
    A = rng.normal(size=(2, 2))
    A = A + A.T
    phi = 0.3 + a[0] * x + a[1] * y + A[0, 0] * x * x + 2 * A[0, 1] * x * y + A[1, 1] * y * y
    grad, lap = orc.gradient_laplacian(p, 9, phi)
    inner = (slice(None), slice(1, -1), slice(1, -1))
    assert np.abs(grad[0][inner] - (a[0] + 2 * (A[0, 0] * x + A[0, 1] * y))[inner]).max() < 1e-9
    assert np.abs(grad[1][inner] - (a[1] + 2 * (A[0, 1] * x + A[1, 1] * y))[inner]).max() < 1e-9
    assert np.abs(grad[2]).max() == 0.0
    assert np.abs(lap[inner] - 2 * (A[0, 0] + A[1, 1])).max() < 1e-9


def test_d2q9_phase_collision_moments(orc):
    rng = np.random.default_rng(22)
    prob = W.Problem(4, 4, 1, q_hydro=9, q_phase=9, xi=4.0, mobility=0.03)
    p = orc.make_problem(prob)
    omega = orc.derived(p)["omega_phi"]
    e, w, _ = orc.lattice(9)
    for _ in range(5):
        h = rng.uniform(0, 0.2, 9)
        u = np.append(rng.normal(0, 0.05, 2), 0.0)
        phic = rng.uniform(0.1, 0.9)
        a = np.append(rng.normal(size=2), 0.0)
        nbprev = I.nb_from_function(lambda d: phic + a @ d)
        hs, phi = orc.phase_cell(p, h, nbprev, u)
        assert hs.sum() == pytest.approx(phi, abs=1e-14) and phi == pytest.approx(h.sum(), abs=1e-15)
        n = a / np.linalg.norm(a)
        theta = (1 - 4 * (phic - 0.5) ** 2) / prob.xi
        exp1 = (1 - omega) * (h @ e) + omega * phi * u + (1 - omega / 2) * CS2 * theta * n
        assert np.abs(hs @ e - exp1).max() < 1e-14
        m2 = np.einsum("i,ia,ib->ab", h, e, e)
        exp2 = (1 - omega) * m2 + omega * phi * (CS2 * D2 + np.outer(u, u))
        assert np.abs(np.einsum("i,ia,ib->ab", hs, e, e) - exp2).max() < 1e-14


def test_d2q9_hydro_collision_moments(orc):
    rng = np.random.default_rng(23)
    prob = W.Problem(4, 4, 1, q_hydro=9, q_phase=9, rho_ratio=50.0, mu_ratio=20.0, sigma=3e-3, xi=4.0,
                     gravity=(1e-4, -2e-4, 0.0), rho_ref=0.7)
    p = orc.make_problem(prob)
    e, w, _ = orc.lattice(9)
    H = np.einsum("ia,ib->iab", e, e) - CS2 * D2[None]
    for _ in range(5):
        g = rng.normal(0, 0.01, 9)
        phic = rng.uniform(0.1, 0.9)
        a = np.append(rng.normal(0, 0.05, 2), 0.0)
        A = np.zeros((3, 3))
        A[:2, :2] = rng.normal(0, 0.02, (2, 2))
        A = A + A.T
        nb = I.nb_from_function(lambda d: phic + a @ d + d @ A @ d)
        gs, u, aux = orc.hydro_cell(p, g, nb)
        rho, pstar, s_nu = aux[0], aux[1], aux[2]
        F = aux[4:7]
        assert F[2] == 0.0 and u[2] == 0.0
        assert pstar == pytest.approx(g.sum(), abs=1e-15) and gs.sum() == pytest.approx(pstar, abs=1e-14)
        assert np.abs(u - (g @ e + F / (2 * rho))).max() < 1e-15
        assert np.abs(gs @ e - (u + F / (2 * rho))).max() < 1e-14
        a2 = np.einsum("i,iab->ab", g, H)
        a2s = np.einsum("i,iab->ab", gs, H)
        assert np.abs(a2s - ((1 - s_nu) * a2 + s_nu * np.outer(u, u))).max() < 1e-14
        # degree <= 2 in the plane: g*/w = c0 + c . e + quadratic(e_x, e_y)
        X = np.column_stack([np.ones(9), e[:, :2], e[:, 0] ** 2, e[:, 1] ** 2, e[:, 0] * e[:, 1]])
        coef, *_ = np.linalg.lstsq(X, gs / w, rcond=None)
        assert np.abs(X @ coef - gs / w).max() < 1e-13


@pytest.mark.parametrize("wall", [(0, 0, 0), (1, 0, 0), (1, 1, 0)])
def test_d2q9_mass_conservation(orc, wall):
    prob = W.Problem(11, 9, 1, wall=wall, q_hydro=9, q_phase=9, rho_ratio=100.0, sigma=5e-4,
                     gravity=(0, -1e-5, 0), rho_ref=0.5)
    s = orc.State(orc.make_problem(prob), W.random_smooth_field(prob.shape, np.random.default_rng(24)))
    m0 = s.phi().sum()
    s.run(40)
    assert abs(s.phi().sum() - m0) <= 1e-12 * m0


def test_d2q9_diffusion_rate(orc):
    prob = W.Problem(64, 1, 1, q_hydro=9, q_phase=9, rho_ratio=1.0, mu_ratio=1.0, nu_H=0.1, sigma=0.0, xi=1e9,
                     mobility=0.05)
    x = np.arange(64) + 0.5
    k = 2 * np.pi / 64
    s = orc.State(orc.make_problem(prob), (0.5 + 0.1 * np.sin(k * x)).reshape(1, 1, 64))
    amps = []
    for T in (500, 2500):
        s.run(T - s.k)
        amps.append(np.sum((s.phi()[0, 0] - 0.5) * np.sin(k * x)))
    assert np.log(amps[0] / amps[1]) / 2000 == pytest.approx(prob.mobility * k * k, rel=5e-3)


def test_d2q9_shear_wave_viscosity(orc):
    phi_u = 0.3
    prob = W.Problem(1, 64, 1, q_hydro=9, q_phase=9)
    y = np.arange(64) + 0.5
    k = 2 * np.pi / 64
    s = orc.State(orc.make_problem(prob), np.full((1, 64, 1), phi_u))
    u = np.zeros((3, 1, 64, 1))
    u[0, 0, :, 0] = 1e-3 * np.sin(k * y)
    Ph._equilibrium_flow(orc, s, prob, u)
    amps = []
    for T in (200, 2200):
        s.run(T - s.k)
        amps.append(np.sum(s.fields()[1][0, 0, :, 0] * np.sin(k * y)))
    tau = 3 * prob.nu_L + phi_u * (3 * prob.nu_H - 3 * prob.nu_L)
    assert np.log(amps[0] / amps[1]) / 2000 == pytest.approx(tau * CS2 * k * k, rel=5e-3)


def test_d2q9_planar_interface_steady(orc):
    prob = W.Problem(64, 1, 1, q_hydro=9, q_phase=9)
    phi0 = W.slab_phi(prob, 16.0, 48.0)
    s = orc.State(orc.make_problem(prob), phi0)
    s.run(2000)
    phi, u, _ = s.fields()
    assert np.abs(phi - phi0).max() < 1e-2 and np.abs(u).max() < 1e-6


def test_d2q9_laplace_law_cylinder(orc):
    sigma = 1e-3
    pts = [Ph._laplace_cylinder(orc, R, sigma=sigma, q=9, qp=9) for R in (8.0, 11.0, 14.0)]
    slope = np.polyfit([1 / r for r, _, _ in pts], [d for _, d, _ in pts], 1)[0]
    assert slope == pytest.approx(sigma, rel=5e-2)
    assert all(umax < 1e-5 for _, _, umax in pts)
