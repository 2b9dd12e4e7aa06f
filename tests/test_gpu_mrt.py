"""The MRT phase-field collision of Section 3.1 (first-order moments relaxed with
omega_phi, all others with 1; weighted-orthogonal basis) on the GPU against the
FP64 oracle, whose MRT step is pinned by a literal M^-1 S M construction, in the
one-cell and the two-cell fused steps.  Tolerances as for the SRT form: relative
L-infinity 1e-5."""
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


# odd nx: the one-cell step; even nx: the two-cell step (the library's choice and
# forced), with one to three tiles along x, a ragged tail, nx = 2 and walls
@pytest.mark.parametrize("form,nx,ny,nz,wall,q", [
    ("fused", 37, 29, 19, (0, 0, 0), 19), ("fused", 33, 17, 11, (1, 1, 1), 27), ("fused", 1, 33, 1, (0, 1, 0), 27),
    ("fused", 38, 29, 19, (0, 0, 0), 19), ("pair", 34, 17, 11, (1, 1, 1), 27), ("pair", 130, 9, 7, (1, 0, 1), 27),
    ("pair", 2, 33, 1, (0, 1, 0), 27), ("cell", 34, 17, 11, (1, 1, 1), 27)])
def test_two_steps_from_random_state(lbm, orc, form, nx, ny, nz, wall, q):
    prob = W.Problem(nx, ny, nz, wall=wall, q_hydro=q, rho_ratio=100.0, mu_ratio=30.0, sigma=1e-3, xi=3.0,
                     mobility=0.07, gravity=(1e-5, -2e-5, 3e-6), rho_ref=0.4, phase_mrt=1)
    h, g, phi = W.random_state(prob, seed=nx * 7 + ny + nz)
    sim = lbm.Simulation.from_problem(prob, form=form)
    sim.set_state(h, g, phi)
    p = orc.make_problem(prob)
    rh, rg, rphi = h.astype(np.float64), g.astype(np.float64), phi.astype(np.float64)
    for step in (1, 2):
        sim.step(1)
        sim.synchronize()
        rg, u = orc.hydro_step(p, rg, rphi)
        rh, rphi = orc.phase_step(p, rh, rphi, u)
        h1, g1, phi1 = sim.get_state()
        assert rel_linf(phi1, rphi) <= TOL, step
        assert rel_linf(h1, rh) <= TOL, step
        assert rel_linf(g1, rg) <= TOL, step
    # and it is not the SRT step
    srt = lbm.Simulation.from_problem(W.Problem(**{**prob.__dict__, "phase_mrt": 0}), form=form)
    srt.set_state(h, g, phi)
    srt.step(2)
    assert np.abs(srt.get_state()[0] - h1).max() > 1e-4


@pytest.mark.parametrize("form", ["fused", "cell"])
def test_static_droplet_200_steps(lbm, orc, form):
    prob, phi0 = W.static_droplet()
    prob.phase_mrt = 1
    sim = lbm.Simulation.from_problem(prob, form=form)
    sim.init_phase(phi0)
    sim.step(200)
    sim.synchronize()
    phi, u, p = (t.cpu().numpy().astype(np.float64) for t in sim.fields())
    ref = orc.State(orc.make_problem(prob), phi0).run(200)
    rphi, ru, rp = ref.fields()
    assert rel_linf(phi, rphi) <= TOL
    assert rel_linf(u, ru, 1e-6) <= TOL
    assert rel_linf(p, rp) <= TOL
    assert abs(phi.sum() / phi0.astype(np.float64).sum() - 1.0) <= 1e-6
