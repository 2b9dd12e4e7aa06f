"""Brute-force pin of the oracle's whole time step on small periodic boxes.

An independent, literal numpy implementation of one step of Section 3:

* neighbours by ``np.roll`` (not the oracle's index arithmetic);
* the hydrodynamic collision in moment space exactly as eq:improved_collision
  writes it, g* = M^{-1} [m - S (m - m^eq + F_m / 2) + F_m], with M built by
  w-weighted Gram-Schmidt of the monomials in degree order (the "weighted
  orthogonal moment set" of Section 6.1), S = diag(1, 1, 1, 1, s_nu x 6, 1, ...),
  F_m = rho^{-1} (0, F, 0, ...);
* the viscous force eq:viscousForce with the collision matrix Omega = M^{-1} S M
  applied to (g - g^eq) literally;
* the phase-field update eq:lb_interface with Omega = omega_phi I.

It shares nothing with the oracle's closed (Hermite) form of the collision, so a
wrong coefficient, sign or index in that reduction fails here.
"""
import itertools

import numpy as np
import pytest

import workloads as W

CS2 = 1.0 / 3.0


def moment_matrix(e, w):
    """Rows: w-orthogonal polynomials of e, Gram-Schmidt in degree order;
    returns (M, degree of each row)."""
    q = len(w)
    exps = sorted(itertools.product(range(3), repeat=3), key=lambda t: (sum(t), [-v for v in t]))
    rows, degs = [], []
    for a, b, c in exps:
        v = (e[:, 0] ** a * e[:, 1] ** b * e[:, 2] ** c).astype(float)
        for r in rows:
            v = v - (w @ (v * r)) / (w @ (r * r)) * r
        if w @ (v * v) > 1e-10:
            rows.append(v)
            degs.append(a + b + c)
        if len(rows) == q:
            break
    M = np.array(rows)
    assert M.shape == (q, q)
    return M, np.array(degs)


def shifted(f, d):
    """f(x + d) on a periodic box, f of shape (nz, ny, nx), d = (dx, dy, dz)."""
    return np.roll(f, shift=(-d[2], -d[1], -d[0]), axis=(0, 1, 2))


def literal_step(prob, orc, h, g, phi_prev, u_prev):
    qp = prob.q_phase
    e15, w15, _ = orc.lattice(qp)
    e, w, _ = orc.lattice(prob.q_hydro)
    q = len(w)
    tau_H, tau_L = prob.nu_H / CS2, prob.nu_L / CS2
    omega = 1.0 / (prob.mobility / CS2 + 0.5)
    beta, kappa = 12 * prob.sigma / prob.xi, 1.5 * prob.sigma * prob.xi

    # ---- phase step
    phi = h.sum(0)
    G = sum(e15[i][:, None, None, None] * w15[i] * shifted(phi_prev, e15[i]) for i in range(qp)) / CS2
    Gn = np.sqrt((G ** 2).sum(0))
    n = np.where(Gn ** 2 > 1e-24, G / np.where(Gn > 0, Gn, 1), 0.0)
    theta = (1 - 4 * (phi_prev - 0.5) ** 2) / prob.xi
    uu = (u_prev ** 2).sum(0)
    h_next = np.zeros_like(h)
    for i in range(qp):
        eu = np.einsum("a,a...->...", e15[i].astype(float), u_prev)
        Gam = w15[i] * (1 + eu / CS2 + eu ** 2 / (2 * CS2 ** 2) - uu / (2 * CS2))
        F = theta * w15[i] * np.einsum("a,a...->...", e15[i].astype(float), n)
        hs = omega * (phi * Gam - h[i] - 0.5 * F) + h[i] + F
        h_next[i] = shifted(hs, -e15[i])

    # ---- hydro step on Phi^k = phi
    M, deg = moment_matrix(e, w)
    Minv = np.linalg.inv(M)
    grad = sum(e[i][:, None, None, None] * w[i] * shifted(phi, e[i]) for i in range(q)) / CS2
    lap = 2 * sum(w[i] * (shifted(phi, e[i]) - phi) for i in range(q)) / CS2
    rho = prob.rho_L + phi * (prob.rho_H - prob.rho_L)
    grad_rho = (prob.rho_H - prob.rho_L) * grad
    tau = tau_L + phi * (tau_H - tau_L)
    s_nu = 1 / (tau + 0.5)
    mu = 4 * beta * phi * (phi - 1) * (phi - 0.5) - kappa * lap
    pstar = g.sum(0)
    F_p = -pstar * CS2 * grad_rho
    F_s = mu * grad
    F_b = (rho - prob.rho_ref)[None] * np.array(prob.gravity, dtype=float)[:, None, None, None]
    j = np.einsum("ia,i...->a...", e.astype(float), g)

    def geq(u):
        uu = (u ** 2).sum(0)
        out = []
        for i in range(q):
            eu = np.einsum("a,a...->...", e[i].astype(float), u)
            Gam = w[i] * (1 + eu / CS2 + eu ** 2 / (2 * CS2 ** 2) - uu / (2 * CS2))
            out.append(pstar * w[i] + (Gam - w[i]))
        return np.array(out)

    rates = lambda s: np.where(deg[:, None, None, None] == 2, s[None], 1.0)  # noqa: E731
    S = rates(s_nu)
    up = j + (F_p + F_s + F_b) / (2 * rho)
    m = np.einsum("ki,i...->k...", M, g)
    neq = np.einsum("ik,k...->i...", Minv, S * (m - np.einsum("ki,i...->k...", M, geq(up))))
    Pi = np.einsum("ia,ib,i...->ab...", e.astype(float), e.astype(float), neq)
    nu = tau * CS2
    F_mu = -(nu / CS2) * np.einsum("ab...,b...->a...", Pi, grad_rho)
    F = F_p + F_s + F_mu + F_b
    u = j + F / (2 * rho)
    m_eq = np.einsum("ki,i...->k...", M, geq(u))
    F_m = np.zeros_like(m)
    first = np.flatnonzero(deg == 1)  # the x, y (, z) rows, in that order
    F_m[first] = (F / rho)[:len(first)]
    m_star = m - S * (m - m_eq + 0.5 * F_m) + F_m
    gs = np.einsum("ik,k...->i...", Minv, m_star)
    g_next = np.array([shifted(gs[i], -e[i]) for i in range(q)])
    return h_next, phi, g_next, u


@pytest.mark.parametrize("q,qp,nz", [(19, 15, 5), (27, 15, 5), (19, 19, 5), (27, 27, 5), (9, 9, 1)])
def test_literal_moment_space_step(orc, q, qp, nz):
    gz = 1e-5 if nz > 1 else 0.0  # a two-dimensional lattice carries no z momentum
    prob = W.Problem(7, 6, nz, wall=(0, 0, 0), q_hydro=q, q_phase=qp, rho_ratio=100.0, mu_ratio=30.0, sigma=2e-3,
                     xi=3.0, mobility=0.03, gravity=(2e-5, -3e-5, gz), rho_ref=0.4)
    p = orc.make_problem(prob)
    rng = np.random.default_rng(11)
    phi_prev = W.random_smooth_field(prob.shape, rng)
    h = rng.uniform(0, 0.1, (qp,) + prob.shape)
    g = rng.normal(0, 1e-3, (q,) + prob.shape)
    u_prev = rng.normal(0, 1e-2, (3,) + prob.shape)

    h_lit, phi_lit, g_lit, u_lit = literal_step(prob, orc, h, g, phi_prev, u_prev)
    h_next, phi_now = orc.phase_step(p, h, phi_prev, u_prev)
    g_next, u_now = orc.hydro_step(p, g, phi_now)

    assert np.abs(phi_now - phi_lit).max() < 1e-14
    assert np.abs(h_next - h_lit).max() < 1e-14
    assert np.abs(u_now - u_lit).max() < 1e-13 * max(1.0, np.abs(u_lit).max())
    assert np.abs(g_next - g_lit).max() < 1e-13 * np.abs(g_lit).max()


def test_moment_matrix_is_weighted_orthogonal(orc):
    for q in (9, 15, 19, 27):
        e, w, _ = orc.lattice(q)
        M, deg = moment_matrix(e, w)
        N = M @ np.diag(w) @ M.T
        assert np.abs(N - np.diag(np.diag(N))).max() < 1e-12
        if q == 9:
            assert list(deg) == [0, 1, 1, 2, 2, 2, 3, 3, 4]
        else:
            assert list(deg[:10]) == [0, 1, 1, 1, 2, 2, 2, 2, 2, 2]


def literal_phase_mrt_step(prob, orc, h, phi_prev, u_prev):
    """eq:lb_interface with Omega = M^{-1} S M literally (Section 3.1): M the
    w-orthogonal moment matrix of the phase lattice, S relaxing the first-order
    moments with omega_phi and every other moment with 1."""
    qp = prob.q_phase
    e15, w15, _ = orc.lattice(qp)
    omega = 1.0 / (prob.mobility / CS2 + 0.5)
    M, deg = moment_matrix(e15, w15)
    Omega = np.linalg.inv(M) @ np.diag(np.where(deg == 1, omega, 1.0)) @ M
    phi = h.sum(0)
    G = sum(e15[i][:, None, None, None] * w15[i] * shifted(phi_prev, e15[i]) for i in range(qp)) / CS2
    Gn = np.sqrt((G ** 2).sum(0))
    n = np.where(Gn ** 2 > 1e-24, G / np.where(Gn > 0, Gn, 1), 0.0)
    theta = (1 - 4 * (phi_prev - 0.5) ** 2) / prob.xi
    uu = (u_prev ** 2).sum(0)
    heq, F = np.zeros_like(h), np.zeros_like(h)
    for i in range(qp):
        eu = np.einsum("a,a...->...", e15[i].astype(float), u_prev)
        heq[i] = phi * w15[i] * (1 + eu / CS2 + eu ** 2 / (2 * CS2 ** 2) - uu / (2 * CS2))
        F[i] = theta * w15[i] * np.einsum("a,a...->...", e15[i].astype(float), n)
    hs = h + np.einsum("ij,j...->i...", Omega, heq - h - 0.5 * F) + F
    return np.array([shifted(hs[i], -e15[i]) for i in range(qp)]), phi


@pytest.mark.parametrize("qp", [15, 19, 27])
def test_literal_mrt_phase_step(orc, qp):
    prob = W.Problem(7, 6, 5, wall=(0, 0, 0), q_hydro=27, q_phase=qp, sigma=2e-3, xi=3.0, mobility=0.07,
                     phase_mrt=1)
    p = orc.make_problem(prob)
    rng = np.random.default_rng(12)
    phi_prev = W.random_smooth_field(prob.shape, rng)
    h = rng.uniform(0, 0.1, (qp,) + prob.shape)
    u_prev = rng.normal(0, 1e-2, (3,) + prob.shape)
    h_lit, phi_lit = literal_phase_mrt_step(prob, orc, h, phi_prev, u_prev)
    h_next, phi_now = orc.phase_step(p, h, phi_prev, u_prev)
    assert np.abs(phi_now - phi_lit).max() < 1e-14
    assert np.abs(h_next - h_lit).max() < 1e-14
    # the MRT step differs from the SRT step (the higher moments relax with 1)
    h_srt, _ = orc.phase_step(orc.make_problem(prob, phase_mrt=0), h, phi_prev, u_prev)
    assert np.abs(h_srt - h_lit).max() > 1e-3


def test_mrt_phase_with_unit_rate_is_srt(orc):
    """omega_phi = 1 (M = c_s^2 / 2) relaxes every moment with 1: MRT == SRT."""
    prob = W.Problem(6, 5, 4, wall=(1, 0, 0), q_hydro=19, sigma=1e-3, xi=3.0, mobility=CS2 / 2)
    rng = np.random.default_rng(13)
    phi_prev = W.random_smooth_field(prob.shape, rng)
    h = rng.uniform(0, 0.1, (15,) + prob.shape)
    u_prev = rng.normal(0, 1e-2, (3,) + prob.shape)
    a, _ = orc.phase_step(orc.make_problem(prob, phase_mrt=1), h, phi_prev, u_prev)
    b, _ = orc.phase_step(orc.make_problem(prob, phase_mrt=0), h, phi_prev, u_prev)
    assert np.abs(a - b).max() < 1e-15
