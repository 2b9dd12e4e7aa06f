"""The two-dimensional pair (D2Q9 phase field + D2Q9 hydrodynamics on an
nx x ny x 1 box, Section 5.1) on the GPU against the FP64 oracle, with the
tolerances of the benchmarked pair."""
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


@pytest.mark.parametrize("nx,ny,wall", [(37, 29, (0, 0, 0)), (33, 17, (1, 1, 0)), (70, 9, (0, 1, 0)),
                                        (38, 29, (0, 0, 0)), (130, 17, (1, 1, 0)), (2, 11, (1, 0, 0))])
def test_two_steps_from_random_state(lbm, orc, nx, ny, wall):
    prob = W.Problem(nx, ny, 1, wall=wall, q_hydro=9, q_phase=9, rho_ratio=100.0, mu_ratio=30.0, sigma=1e-3,
                     xi=3.0, mobility=0.03, gravity=(1e-5, -2e-5, 0.0), rho_ref=0.4)
    h, g, phi = W.random_state(prob, seed=nx + ny)
    sim = lbm.Simulation.from_problem(prob)
    sim.set_state(h, g, phi)
    p = orc.make_problem(prob)
    rh, rg, rphi = h.astype(np.float64), g.astype(np.float64), phi.astype(np.float64)
    for step in (1, 2):
        sim.step(1)
        sim.synchronize()
        rg, u = orc.hydro_step(p, rg, rphi)
        rh, rphi = orc.phase_step(p, rh, rphi, u)
        h1, g1, phi1 = sim.get_state()
        assert h1.shape[0] == 9 and g1.shape[0] == 9
        assert rel_linf(phi1, rphi) <= TOL, step
        assert rel_linf(h1, rh) <= TOL, step
        assert rel_linf(g1, rg) <= TOL, step


@pytest.mark.parametrize("form", ["fused", "cell"])
def test_droplet_200_steps(lbm, orc, form):
    prob = W.Problem(48, 48, 1, q_hydro=9, q_phase=9, rho_ratio=1000.0, nu_H=0.01, mu_ratio=100.0, sigma=1e-4,
                     xi=5.0, mobility=0.02)
    phi0 = W.cylinder_phi(prob, (24.0, 24.0), 10.0, heavy_inside=True).astype(np.float32)
    sim = lbm.Simulation.from_problem(prob, form=form)
    sim.init_phase(phi0)
    sim.step(200)
    sim.synchronize()
    phi, u, p = (t.cpu().numpy().astype(np.float64) for t in sim.fields())
    rphi, ru, rp = orc.State(orc.make_problem(prob), phi0).run(200).fields()
    assert rel_linf(phi, rphi) <= TOL
    assert rel_linf(u, ru, 1e-6) <= TOL
    assert rel_linf(p, rp) <= TOL
    assert np.abs(u[2]).max() == 0.0
    d = sim.reduce()
    assert abs(d["mass"] / phi0.astype(np.float64).sum() - 1.0) <= 1e-6
    assert d["mass"] == pytest.approx(phi.sum(), rel=1e-9)


def test_benchmark_box_sample(lbm):
    """A 512 x 1024 cut of the two-dimensional benchmark recipe: 100 steps stay
    finite, mass kept."""
    prob, phi0 = W.roofline2d(512, 1024)
    sim = lbm.Simulation.from_problem(prob)
    sim.init_phase(phi0)
    m0 = sim.reduce()["mass"]
    sim.step(100)
    sim.synchronize()
    assert abs(sim.reduce()["mass"] / m0 - 1.0) <= 1e-6
