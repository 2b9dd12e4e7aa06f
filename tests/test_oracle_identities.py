"""Pins of the FP64 oracle against closed forms and invariants fixed by the paper.

* lattice moment identities of D3Q15 / D3Q19 / D3Q27 (the isotropy that the
  stencils eq:grad, eq:lap and the equilibria of Section 3 rely on);
* eq:grad / eq:lap are exact on linear and quadratic fields;
* collision moments: sum h* = phi, first and second moments of h* and g*
  follow from h^eq = phi Gamma_i, g^eq = p* w_i + (Gamma_i - w_i),
  eq:interfaceTracking and eq:improved_collision (closed forms derived from
  moment algebra, not per-direction formulas);
* exact conservation of sum phi (conservative Allen-Cahn equation) on periodic
  and walled boxes; trivial states stay unchanged.
"""
import numpy as np
import pytest

import workloads as W

CS2 = 1.0 / 3.0


def nb_from_function(f):
    """3x3x3 neighbourhood array nb[(dz+1)*9+(dy+1)*3+(dx+1)] = f(dx, dy, dz)."""
    nb = np.zeros(27)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                nb[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)] = f(np.array([dx, dy, dz], dtype=float))
    return nb


@pytest.mark.parametrize("q", [15, 19, 27])
def test_lattice_moments(orc, q):
    e, w, opp = orc.lattice(q)
    assert len(w) == q and len({tuple(v) for v in e}) == q
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs((w[:, None] * e).sum(0)).max() < 1e-15
    m2 = np.einsum("i,ia,ib->ab", w, e, e)
    assert np.abs(m2 - CS2 * np.eye(3)).max() < 1e-15
    m3 = np.einsum("i,ia,ib,ic->abc", w, e, e, e)
    assert np.abs(m3).max() < 1e-15
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, e, e, e, e)
    d = np.eye(3)
    iso = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d))
    assert np.abs(m4 - iso).max() < 1e-15
    assert (e[opp] == -e).all()
    # numbering: rest first, each moving direction followed by its opposite
    assert (e[0] == 0).all()
    for i in range(1, q, 2):
        assert opp[i] == i + 1 and opp[i + 1] == i


@pytest.mark.parametrize("q", [15, 19, 27])
def test_stencils_exact_on_quadratics(orc, q):
    rng = np.random.default_rng(1)
    prob = W.Problem(12, 10, 9, wall=(0, 0, 0), q_hydro=19)
    p = orc.make_problem(prob)
    z, y, x = np.meshgrid(np.arange(9.0), np.arange(10.0), np.arange(12.0), indexing="ij")
    X = np.stack([x, y, z])
    a = rng.normal(size=3)
    A = rng.normal(size=(3, 3))
    A = A + A.T
    phi = 0.3 + np.einsum("a,a...->...", a, X) + np.einsum("ab,a...,b...->...", A, X, X)
    grad, lap = orc.gradient_laplacian(p, q, phi)
    inner = (slice(1, -1),) * 3  # the wrap seam of a periodic box is not polynomial
    exact_grad = a[:, None, None, None] + 2 * np.einsum("ab,b...->a...", A, X)
    assert np.abs(grad[(slice(None),) + inner] - exact_grad[(slice(None),) + inner]).max() < 1e-9
    assert np.abs(lap[inner] - 2 * np.trace(A)).max() < 1e-9


def test_stencil_walls_mirror(orc):
    """On a walled axis the ghost value repeats the first interior cell, so a
    field that is constant along the wall normal has zero normal gradient."""
    prob = W.Problem(6, 7, 5, wall=(1, 1, 1), q_hydro=27)
    p = orc.make_problem(prob)
    rng = np.random.default_rng(2)
    phi = np.broadcast_to(rng.uniform(size=(1, 1, 6)), (5, 7, 6)).copy()  # varies along x only
    grad, lap = orc.gradient_laplacian(p, 27, phi)
    assert np.abs(grad[1]).max() < 1e-15 and np.abs(grad[2]).max() < 1e-15
    # mirrored ghosts: gradient at x = 0 uses phi(-1) = phi(0)
    g0 = grad[0][:, :, 0]
    assert np.allclose(g0, 0.5 * (phi[:, :, 1] - phi[:, :, 0]), atol=1e-14)


def test_derived_parameters(orc):
    prob, _ = W.static_droplet()
    d = orc.derived(orc.make_problem(prob))
    assert d["tau_H"] == pytest.approx(0.03) and d["tau_L"] == pytest.approx(0.3)
    assert d["omega_phi"] == pytest.approx(1.0 / (3 * 0.02 + 0.5))
    assert d["beta"] == pytest.approx(12e-4 / 5) and d["kappa"] == pytest.approx(1.5e-4 * 5)


@pytest.mark.parametrize("qp", [15, 19, 27])
def test_phase_collision_moments(orc, qp):
    """sum h* = phi; first/second moments from relaxation toward phi Gamma(u)
    plus the interface forcing, whose zeroth and second moments vanish and
    whose first moment is c_s^2 theta n (lattice isotropy), on each phase lattice."""
    rng = np.random.default_rng(3)
    prob = W.Problem(4, 4, 4, xi=4.0, mobility=0.03, q_phase=qp)
    p = orc.make_problem(prob)
    omega = orc.derived(p)["omega_phi"]
    e, w, _ = orc.lattice(qp)
    for trial in range(5):
        h = rng.uniform(0, 0.2, qp)
        u = rng.normal(0, 0.05, 3)
        phic = rng.uniform(0.1, 0.9)
        a = rng.normal(size=3)
        nbprev = nb_from_function(lambda d: phic + a @ d)  # linear: gradient exactly a
        hs, phi = orc.phase_cell(p, h, nbprev, u)
        assert phi == pytest.approx(h.sum(), abs=1e-15)
        assert hs.sum() == pytest.approx(phi, abs=1e-14)
        n = a / np.linalg.norm(a)
        theta = (1 - 4 * (phic - 0.5) ** 2) / prob.xi
        m1 = h @ e
        exp1 = (1 - omega) * m1 + omega * phi * u + (1 - omega / 2) * CS2 * theta * n
        assert np.abs(hs @ e - exp1).max() < 1e-14
        m2 = np.einsum("i,ia,ib->ab", h, e, e)
        exp2 = (1 - omega) * m2 + omega * phi * (CS2 * np.eye(3) + np.outer(u, u))
        assert np.abs(np.einsum("i,ia,ib->ab", hs, e, e) - exp2).max() < 1e-14


@pytest.mark.parametrize("qp", [15, 19, 27])
def test_phase_normal_zero_gradient(orc, qp):
    """A flat neighbourhood has no normal: the forcing vanishes and h relaxes to phi Gamma(u)."""
    prob = W.Problem(4, 4, 4, q_phase=qp)
    p = orc.make_problem(prob)
    omega = orc.derived(p)["omega_phi"]
    e, w, _ = orc.lattice(qp)
    h = np.full(qp, 0.05)
    hs, phi = orc.phase_cell(p, h, np.full(27, 0.5), np.zeros(3))
    assert np.allclose(hs, (1 - omega) * h + omega * phi * w, atol=1e-15)


@pytest.mark.parametrize("q", [19, 27])
def test_hydro_collision_moments(orc, q):
    """Zeroth moment p* kept; first moment u + F/(2 rho) with u = j + F/(2 rho);
    Hermite second moment (1 - s_nu) a2 + s_nu u u (eq:improved_collision with the
    force in the first moments only)."""
    rng = np.random.default_rng(4)
    prob = W.Problem(4, 4, 4, q_hydro=q, rho_ratio=50.0, mu_ratio=20.0, sigma=3e-3, xi=4.0,
                     gravity=(1e-4, -2e-4, 3e-5), rho_ref=0.7)
    p = orc.make_problem(prob)
    e, w, _ = orc.lattice(q)
    for trial in range(5):
        g = rng.normal(0, 0.01, q)
        phic = rng.uniform(0.1, 0.9)
        a = rng.normal(0, 0.05, 3)
        A = rng.normal(0, 0.02, (3, 3))
        A = A + A.T
        nb = nb_from_function(lambda d: phic + a @ d + d @ A @ d)  # grad = a, lap = 2 tr A
        gs, u, aux = orc.hydro_cell(p, g, nb)
        rho, pstar, s_nu, tau = aux[0], aux[1], aux[2], aux[3]
        F = aux[4:7]
        assert rho == pytest.approx(prob.rho_L + phic * (prob.rho_H - prob.rho_L))
        assert pstar == pytest.approx(g.sum(), abs=1e-15)
        j = g @ e
        assert np.abs(u - (j + F / (2 * rho))).max() < 1e-15
        assert gs.sum() == pytest.approx(pstar, abs=1e-14)
        assert np.abs(gs @ e - (u + F / (2 * rho))).max() < 1e-14
        H = np.einsum("ia,ib->iab", e, e) - CS2 * np.eye(3)[None]
        a2 = np.einsum("i,iab->ab", g, H)
        a2s = np.einsum("i,iab->ab", gs, H)
        assert np.abs(a2s - ((1 - s_nu) * a2 + s_nu * np.outer(u, u))).max() < 1e-14
        # nothing of degree >= 3 survives: g*/w is a polynomial of degree <= 2 in e
        X = np.column_stack([np.ones(q), e, e[:, 0] ** 2, e[:, 1] ** 2, e[:, 2] ** 2,
                             e[:, 0] * e[:, 1], e[:, 0] * e[:, 2], e[:, 1] * e[:, 2]])
        coef, *_ = np.linalg.lstsq(X, gs / w, rcond=None)
        assert np.abs(X @ coef - gs / w).max() < 1e-13
        # tau interpolation and s_nu
        d = orc.derived(p)
        assert tau == pytest.approx(d["tau_L"] + phic * (d["tau_H"] - d["tau_L"]))
        assert s_nu == pytest.approx(1 / (tau + 0.5))


def test_hydro_forces_vanish_in_uniform_phase(orc):
    """Uniform phi: no surface tension, no pressure force, no viscous force; with
    rho_ref = rho the buoyancy vanishes too, so the collision conserves j."""
    prob = W.Problem(4, 4, 4, q_hydro=27, gravity=(0, -1e-3, 0), rho_ref=1.0)
    p = orc.make_problem(prob)
    rng = np.random.default_rng(5)
    g = rng.normal(0, 0.01, 27)
    gs, u, aux = orc.hydro_cell(p, g, np.full(27, 1.0))  # phi = 1: rho = rho_H = rho_ref
    assert np.abs(aux[4:7]).max() < 1e-18
    e, _, _ = orc.lattice(27)
    assert np.abs(gs @ e - g @ e).max() < 1e-15


@pytest.mark.parametrize("wall,q,qp", [((0, 0, 0), 19, 15), ((1, 0, 0), 19, 15), ((1, 1, 1), 19, 15),
                                       ((0, 1, 0), 19, 15), ((0, 0, 0), 27, 15), ((1, 0, 0), 27, 15),
                                       ((1, 1, 1), 27, 15), ((0, 1, 0), 27, 15), ((1, 1, 1), 19, 19),
                                       ((1, 0, 1), 27, 27), ((0, 1, 0), 19, 27)])
def test_mass_conservation(orc, wall, q, qp):
    """sum_x phi is conserved to round-off: sum_i F^phi_i = 0, the collision keeps
    the zeroth moment and streaming / bounce-back only moves populations."""
    prob = W.Problem(11, 9, 7, wall=wall, q_hydro=q, q_phase=qp, rho_ratio=100.0, sigma=5e-4,
                     gravity=(0, -1e-5, 0), rho_ref=0.5)
    p = orc.make_problem(prob)
    rng = np.random.default_rng(6)
    phi0 = W.random_smooth_field(prob.shape, rng)
    s = orc.State(p, phi0)
    m0 = s.phi().sum()
    s.run(40)
    assert abs(s.phi().sum() - m0) <= 1e-12 * m0
    # the hydrodynamic zeroth moment (sum p*) is also conserved by collision and streaming
    s2 = orc.State(p, phi0)
    s2.g[:] = rng.normal(0, 1e-4, s2.g.shape)
    p0 = s2.g.sum()
    s2.run(10)
    assert abs(s2.g.sum() - p0) < 1e-13


@pytest.mark.parametrize("q", [19, 27])
def test_trivial_states(orc, q):
    """Uniform phi at rest with no force: nothing changes.  Uniform phi with a
    uniform velocity and no force: the flow is kept and h stays phi Gamma(u)."""
    prob = W.Problem(6, 5, 4, q_hydro=q, gravity=(0, 0, 0))
    p = orc.make_problem(prob)
    s = orc.State(p, np.full(prob.shape, 0.37))
    h0 = s.h.copy()
    s.run(10)
    assert np.abs(s.h - h0).max() < 1e-15 and np.abs(s.g).max() < 1e-15
    # uniform flow
    e, w, _ = orc.lattice(q)
    eh, wh, _ = orc.lattice(15)
    U = np.array([0.03, -0.02, 0.01])
    s = orc.State(p, np.full(prob.shape, 0.6))
    eu = e @ U
    s.g[:] = (w * (3 * eu + 4.5 * eu ** 2 - 1.5 * U @ U))[:, None, None, None]  # g^eq at p* = 0
    s.u_prev[:] = U[:, None, None, None]
    ehu = eh @ U
    heq = 0.6 * wh * (1 + 3 * ehu + 4.5 * ehu ** 2 - 1.5 * U @ U)
    s.h[:] = heq[:, None, None, None]
    s.run(10)
    phi, u, pr = s.fields()
    assert np.abs(u - U[:, None, None, None]).max() < 1e-14
    assert np.abs(phi - 0.6).max() < 1e-14
    assert np.abs(s.h - heq[:, None, None, None]).max() < 1e-14


@pytest.mark.parametrize("q", [19, 27])
def test_chemical_potential_vanishes_on_equilibrium_profile(orc, q):
    """beta = 12 sigma/xi and kappa = 3 sigma xi/2 make the tanh profile of width
    xi (Section 3.1) the equilibrium of the chemical potential eq:chemPot:
    mu_phi = 0 there, up to the O(1/xi^2) error of the stencil eq:lap."""
    xi = 8.0
    prob = W.Problem(4, 4, 4, q_hydro=q, rho_ratio=1.0, sigma=1e-3, xi=xi)
    p = orc.make_problem(prob)
    beta = 12 * prob.sigma / xi
    n = np.array([1.0, 2.0, 2.0]) / 3.0
    for x0 in np.linspace(-xi, xi, 9):
        nb = nb_from_function(lambda d: 0.5 + 0.5 * np.tanh(2 * (d @ n - x0) / xi))
        _, _, aux = orc.hydro_cell(p, np.zeros(q), nb)
        assert abs(aux[7]) < 1e-2 * beta
