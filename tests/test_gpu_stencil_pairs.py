"""The other stencil pairs (Section 5.1): D3Q19 and D3Q27 phase-field lattices with
D3Q19 or D3Q27 hydrodynamics, FP32, against the FP64 oracle with the same
tolerances as the benchmarked D3Q15 + D3Q27 pair."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5
PAIRS = [(19, 19), (27, 27), (19, 27), (27, 19)]  # (q_phase, q_hydro)


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


@pytest.mark.parametrize("qp,q", PAIRS)
@pytest.mark.parametrize("nx,ny,nz,wall", [(37, 29, 19, (0, 0, 0)), (33, 17, 11, (1, 1, 1)),
                                           (38, 29, 19, (0, 0, 0)), (66, 17, 11, (1, 1, 1))])
def test_two_steps_from_random_state(lbm, orc, qp, q, nx, ny, nz, wall):
    prob = W.Problem(nx, ny, nz, wall=wall, q_hydro=q, q_phase=qp, rho_ratio=100.0, mu_ratio=30.0, sigma=1e-3,
                     xi=3.0, mobility=0.03, gravity=(1e-5, -2e-5, 3e-6), rho_ref=0.4)
    h, g, phi = W.random_state(prob, seed=qp * 100 + q + nx)
    sim = lbm.Simulation.from_problem(prob)
    sim.set_state(h, g, phi)
    assert all(np.array_equal(a, b) for a, b in zip(sim.get_state(), (h, g, phi)))
    p = orc.make_problem(prob)
    rh, rg, rphi = h.astype(np.float64), g.astype(np.float64), phi.astype(np.float64)
    for step in (1, 2):
        sim.step(1)
        sim.synchronize()
        rg, u = orc.hydro_step(p, rg, rphi)
        rh, rphi = orc.phase_step(p, rh, rphi, u)
        h1, g1, phi1 = sim.get_state()
        assert h1.shape[0] == qp
        assert rel_linf(phi1, rphi) <= TOL, step
        assert rel_linf(h1, rh) <= TOL, step
        assert rel_linf(g1, rg) <= TOL, step


@pytest.mark.parametrize("form", ["fused", "cell"])
@pytest.mark.parametrize("qp,q", [(19, 19), (27, 27)])
def test_static_droplet_200_steps(lbm, orc, qp, q, form):
    """32^3 (nx even: the two-cell step by default) and the one-cell step."""
    prob, phi0 = W.static_droplet(q_hydro=q)
    prob.q_phase = qp
    sim = lbm.Simulation.from_problem(prob, form=form)
    sim.init_phase(phi0)
    sim.step(200)
    sim.synchronize()
    phi, u, p = (t.cpu().numpy().astype(np.float64) for t in sim.fields())
    rphi, ru, rp = orc.State(orc.make_problem(prob), phi0).run(200).fields()
    assert rel_linf(phi, rphi) <= TOL
    assert rel_linf(u, ru, 1e-6) <= TOL
    assert rel_linf(p, rp) <= TOL
    assert abs(sim.reduce()["mass"] / phi0.astype(np.float64).sum() - 1.0) <= 1e-6
