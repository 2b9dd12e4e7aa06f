"""GPU (FP32, CUDA library through the C ABI) vs FP64 oracle parity.

Tolerance: relative L-infinity max|a - b| / max|b| <= 1e-5 on phi, u and p
(denominator of u floored at 1e-6, the scale of the spurious currents); phase
mass drift <= 1e-6 relative.  One-step checks from random states compare every
population of both lattices.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2012_06144_gb300 import lbm

    return lbm


def rel_linf(a, b, floor=0.0):
    return float(np.abs(np.asarray(a, np.float64) - b).max() / max(np.abs(b).max(), floor))


def oracle_one_step(orc, prob, h, g, phi):
    """Oracle from the library's state (g^t, h^{t+1}, phi^t): hydro(t) then phase(t+1)."""
    p = orc.make_problem(prob)
    g_next, u = orc.hydro_step(p, g.astype(np.float64), phi.astype(np.float64))
    h_next, phi_next = orc.phase_step(p, h.astype(np.float64), phi.astype(np.float64), u)
    return h_next, g_next, phi_next


@pytest.mark.parametrize("form", ["fused", "cell"])
def test_static_droplet_200_steps(lbm, orc, form):
    """32^3 periodic, D3Q15 + D3Q19, rho ratio 1000, 200 steps; the default fused
    step (two cells per thread on this even box) and the one-cell variant."""
    prob, phi0 = W.static_droplet()
    sim = lbm.Simulation.from_problem(prob, form=form)
    sim.init_phase(phi0)
    m0 = sim.reduce()["mass"]
    sim.step(200)
    sim.synchronize()
    phi, u, p = (t.cpu().numpy() for t in sim.fields())
    m1 = sim.reduce()["mass"]
    ref = orc.State(orc.make_problem(prob), phi0).run(200)
    rphi, ru, rp = ref.fields()
    assert rel_linf(phi, rphi) <= TOL
    assert rel_linf(u, ru, 1e-6) <= TOL
    assert rel_linf(p, rp) <= TOL
    assert abs(m1 - m0) <= 1e-6 * abs(m0)
    assert abs(m1 - rphi.sum()) <= 1e-6 * abs(m0)


CASES = [
    # (nx, ny, nz, wall, q): several tiles and ragged tails in x and y, walls in every combination
    (37, 29, 19, (0, 0, 0), 19),
    (37, 29, 19, (1, 0, 0), 27),
    (37, 29, 19, (0, 1, 1), 19),
    (33, 17, 11, (1, 1, 1), 27),
    (1, 33, 1, (0, 1, 0), 27),
    (64, 8, 3, (0, 0, 1), 19),
    (2, 2, 2, (0, 0, 0), 27),
]


@pytest.mark.parametrize("nx,ny,nz,wall,q", CASES)
def test_one_step_from_random_state(lbm, orc, nx, ny, nz, wall, q):
    prob = W.Problem(nx, ny, nz, wall=wall, q_hydro=q, rho_ratio=100.0, mu_ratio=30.0, sigma=1e-3, xi=3.0,
                     mobility=0.03, gravity=(1e-5, -2e-5, 3e-6), rho_ref=0.4)
    h, g, phi = W.random_state(prob, seed=nx * 1000 + ny * 10 + nz)
    sim = lbm.Simulation.from_problem(prob)
    sim.set_state(h, g, phi)
    sim.step(1)
    sim.synchronize()
    h1, g1, phi1 = sim.get_state()
    rh, rg, rphi = oracle_one_step(orc, prob, h, g, phi)
    assert rel_linf(phi1, rphi) <= TOL
    assert rel_linf(h1, rh) <= TOL
    assert rel_linf(g1, rg) <= TOL


@pytest.mark.parametrize("nx,ny,nz,wall,q", CASES)
def test_two_steps_from_random_state(lbm, orc, nx, ny, nz, wall, q):
    """Covers the second in-place layout of both lattices (g swapped, h natural)."""
    prob = W.Problem(nx, ny, nz, wall=wall, q_hydro=q, rho_ratio=100.0, mu_ratio=30.0, sigma=1e-3, xi=3.0,
                     mobility=0.03, gravity=(1e-5, -2e-5, 3e-6), rho_ref=0.4)
    h, g, phi = W.random_state(prob, seed=nx * 1000 + ny * 10 + nz + 7)
    sim = lbm.Simulation.from_problem(prob)
    sim.set_state(h, g, phi)
    sim.step(2)
    sim.synchronize()
    h2, g2, phi2 = sim.get_state()
    rh, rg, rphi = oracle_one_step(orc, prob, h, g, phi)
    rh, rg, rphi = oracle_one_step(orc, prob, rh, rg, rphi)
    assert rel_linf(phi2, rphi) <= TOL
    assert rel_linf(h2, rh) <= TOL
    assert rel_linf(g2, rg) <= TOL


@pytest.mark.parametrize("steps", [0, 1, 2, 5])
def test_state_roundtrip_each_parity(lbm, steps):
    """set_state followed by get_state returns the input exactly, whatever the
    in-place layout of either lattice."""
    prob = W.Problem(13, 7, 5, wall=(1, 0, 1), q_hydro=27)
    h, g, phi = W.random_state(prob, seed=3)
    sim = lbm.Simulation.from_problem(prob)
    sim.set_state(h, g, phi)
    sim.step(steps)
    h1, g1, phi1 = sim.get_state()
    sim.set_state(h1, g1, phi1)
    h2, g2, phi2 = sim.get_state()
    assert np.array_equal(h1, h2) and np.array_equal(g1, g2) and np.array_equal(phi1, phi2)
    if steps == 0:
        assert np.array_equal(h1, h) and np.array_equal(g1, g) and np.array_equal(phi1, phi)


def test_split_steps_bitwise(lbm):
    prob, phi0 = W.static_droplet(n=20, radius=6.0, q_hydro=27)
    a = lbm.Simulation.from_problem(prob)
    a.init_phase(phi0)
    a.step(9)
    b = lbm.Simulation.from_problem(prob)
    b.init_phase(phi0)
    b.step(4)
    b.step(0)
    b.step(5)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    assert a.steps_done() == b.steps_done() == 9


def test_rising_bubble_walls(lbm, orc):
    """Walled box, D3Q27, gravity, buoyancy and the phi clamp (Eo 10, Mo 1e-3,
    t_ref 1000): 150 steps against the oracle.  phi, u and p within 1e-5, phi on
    the cells with phi < 0.999 (the bubble and its interface).  In the heavy bulk
    the phase step's normal G/|G| follows gradients of the size of the rounding,
    so rounding moves phi there: the FP64 oracle run with its state rounded to
    float32 after every step departs from the plain oracle by 1.1e-5 in phi on
    this case, all of it in the bulk (7e-8 elsewhere); the whole box is held to
    3e-5."""
    prob, phi0 = W.rising_bubble(24, 48, 20, D=12.0, t_ref=1000.0)
    sim = lbm.Simulation.from_problem(prob)
    sim.init_phase(phi0)
    sim.step(150)
    sim.synchronize()
    phi, u, p = sim.fields(on_device=False)
    rphi, ru, rp = orc.State(orc.make_problem(prob), phi0).run(150).fields()
    bubble = rphi < 0.999
    err = np.abs(phi.astype(np.float64) - rphi)
    print("walled 24x48x20, 150 steps: phi (phi < 0.999)", err[bubble].max(), "phi (box)", err.max(),
          "u", rel_linf(u, ru, 1e-6), "p", rel_linf(p, rp))
    assert err[bubble].max() / np.abs(rphi).max() <= TOL
    assert err.max() / np.abs(rphi).max() <= 3e-5
    assert rel_linf(u, ru, 1e-6) <= TOL
    assert rel_linf(p, rp) <= TOL


def test_host_and_device_outputs_agree(lbm):
    prob, phi0 = W.static_droplet(n=16, radius=5.0)
    sim = lbm.Simulation.from_problem(prob)
    sim.init_phase(phi0)
    sim.step(7)
    for d, hst in zip(sim.fields(on_device=True), sim.fields(on_device=False)):
        assert np.array_equal(d.cpu().numpy(), hst)
    for d, hst in zip(sim.get_state(on_device=True), sim.get_state(on_device=False)):
        assert np.array_equal(d.cpu().numpy(), hst)


def test_reduce_matches_fields(lbm):
    prob, phi0 = W.rising_bubble(16, 32, 16, D=8.0, t_ref=200.0)
    sim = lbm.Simulation.from_problem(prob)
    sim.init_phase(phi0)
    sim.step(30)
    phi, u, p = (t.cpu().numpy().astype(np.float64) for t in sim.fields())
    d = sim.reduce()
    rho = prob.rho_L + np.clip(phi, 0, 1) * (prob.rho_H - prob.rho_L)  # the workload clamps phi in rho
    lf = np.clip(1 - 2 * phi, 0, 1)  # bubble indicator
    z, y, x = np.meshgrid(np.arange(16) + .5, np.arange(32) + .5, np.arange(16) + .5, indexing="ij")
    assert d["mass"] == pytest.approx(phi.sum(), rel=1e-9)
    assert d["mom_y"] == pytest.approx((rho * u[1]).sum(), rel=1e-5, abs=1e-12)
    assert d["light_vol"] == pytest.approx(lf.sum(), rel=1e-9)
    assert d["light_y"] == pytest.approx((y * lf).sum() / lf.sum(), rel=1e-9)
    assert d["light_uy"] == pytest.approx((u[1] * lf).sum() / lf.sum(), rel=1e-5, abs=1e-12)
    assert d["max_u"] == pytest.approx(np.sqrt((u ** 2).sum(0)).max(), rel=1e-6)


def test_state_errors(lbm):
    prob, phi0 = W.static_droplet(n=8, radius=2.0)
    sim = lbm.Simulation.from_problem(prob)
    with pytest.raises(lbm.LBMError) as ei:
        sim.step(1)
    assert ei.value.status == lbm.LBM_ERR_STATE
    sim.init_phase(phi0)
    with pytest.raises(lbm.LBMError) as ei:
        sim.step(-1)
    assert ei.value.status == lbm.LBM_ERR_ARG
    sim.step(0)
    assert sim.steps_done() == 0


def test_divergence_is_reported(lbm):
    """A non-finite phi injected from the host comes back as LBM_ERR_DIVERGED."""
    prob, phi0 = W.static_droplet(n=8, radius=2.0)
    phi0 = phi0.copy()
    phi0[3, 4, 5] = np.nan
    sim = lbm.Simulation.from_problem(prob)
    sim.init_phase(phi0)
    sim.step(2)
    with pytest.raises(lbm.LBMError) as ei:
        sim.synchronize()
    assert ei.value.status == lbm.LBM_ERR_DIVERGED
    # a fresh state clears the flag
    sim.init_phase(np.full(prob.shape, 0.5, np.float32))
    sim.step(2)
    sim.synchronize()


@pytest.mark.parametrize("q", [19, 27])
def test_graph_replayed_steps_bitwise(lbm, q):
    """On its own stream a small box replays runs of 16 steps from CUDA graphs
    (one per starting AA parity and phi buffer): 40 steps taken as 16 + 16 + 8
    and as 40 single steps give bit-identical states, from an even and an odd
    level; the level counter follows."""
    import torch

    prob, phi0 = W.static_droplet(n=20, radius=6.0, q_hydro=q)
    stream = torch.cuda.Stream()
    a = lbm.Simulation.from_problem(prob, stream=stream)
    b = lbm.Simulation.from_problem(prob, stream=stream)
    for sim, first in ((a, 1), (b, 1)):
        sim.init_phase(phi0)
        sim.step(first)  # start the runs from an odd level
    a.step(40)  # graphs from levels 1 and 17, then 8 single steps
    a.step(7)
    a.step(26)  # a graph from level 48, then 10 single steps
    for _ in range(73):
        b.step(1)
    a.synchronize()
    b.synchronize()
    assert a.steps_done() == b.steps_done() == 74
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
