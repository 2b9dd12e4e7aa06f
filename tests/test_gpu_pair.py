"""The two-cells-per-thread fused step (LBM_FORM_FUSED_PAIR) against the FP64
oracle, in every storage format.

The pair form moves a population of both cells by one access where the two
locations are neighbours in memory and by one access per cell where they are
not (the swapped lattice's x-moving populations, periodic wrap in x, x walls),
so the cases cover boxes with one, two and three tiles along x, ragged tails,
nx = 2, and walls in every combination; one and two steps reach both AA layouts
of both lattices.  Tolerances: FP32 1e-5 relative on every population (as the
one-cell form); FP16 / BF16 as in test_gpu_precision (each stored moving
population rounds once, the rest population carries the others' rounding).
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5
UNIT = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}


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


def oracle_steps(orc, prob, h, g, phi, n):
    p = orc.make_problem(prob)
    h, g, phi = (a.astype(np.float64) for a in (h, g, phi))
    for _ in range(n):
        g, u = orc.hydro_step(p, g, phi)
        h, phi = orc.phase_step(p, h, phi, u)
    return h, g, phi


CASES = [
    # (nx, ny, nz, wall, q): one x tile with a ragged tail, two and three x tiles, nx = 2
    (38, 29, 19, (0, 0, 0), 27),
    (38, 29, 19, (1, 0, 0), 19),
    (66, 17, 11, (1, 1, 1), 27),
    (66, 9, 7, (0, 1, 1), 19),
    (130, 5, 6, (1, 0, 1), 27),
    (2, 9, 5, (1, 1, 0), 27),
    (2, 4, 3, (0, 0, 0), 19),
    (64, 8, 3, (0, 0, 1), 27),
]


@pytest.mark.parametrize("steps", [1, 2])
@pytest.mark.parametrize("nx,ny,nz,wall,q", CASES)
def test_pair_fp32_from_random_state(lbm, orc, nx, ny, nz, wall, q, steps):
    prob = W.Problem(nx, ny, nz, wall=wall, q_hydro=q, rho_ratio=100.0, mu_ratio=30.0, sigma=1e-3, xi=3.0,
                     mobility=0.03, gravity=(1e-5, -2e-5, 3e-6), rho_ref=0.4)
    h, g, phi = W.random_state(prob, seed=nx * 1000 + ny * 10 + nz + steps)
    sim = lbm.Simulation.from_problem(prob, form="pair")
    sim.set_state(h, g, phi)
    sim.step(steps)
    sim.synchronize()
    h1, g1, phi1 = sim.get_state()
    rh, rg, rphi = oracle_steps(orc, prob, h, g, phi, steps)
    assert rel_linf(phi1, rphi) <= TOL
    assert rel_linf(h1, rh) <= TOL
    assert rel_linf(g1, rg) <= TOL


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("steps", [1, 2])
@pytest.mark.parametrize("nx,ny,nz,wall,q", [CASES[0], CASES[2], CASES[4], CASES[5], CASES[3]])
def test_pair_16bit_from_random_state(lbm, orc, prec, nx, ny, nz, wall, q, steps):
    prob = W.Problem(nx, ny, nz, wall=wall, q_hydro=q, rho_ratio=100.0, mu_ratio=30.0, sigma=1e-3, xi=3.0,
                     mobility=0.03, gravity=(1e-5, -2e-5, 3e-6), rho_ref=0.4, store_phi_ref=0.0)
    h, g, phi = W.random_state(prob, seed=nx + ny + nz + steps)
    sim = lbm.Simulation.from_problem(prob, precision=prec, form="pair")
    sim.set_state(h, g, phi)
    h0, g0, phi0 = sim.get_state()  # the representable state the steps start from
    sim.step(steps)
    sim.synchronize()
    h1, g1, phi1 = sim.get_state()
    rh, rg, rphi = oracle_steps(orc, prob, h0, g0, phi0, steps)
    u = UNIT[prec]
    # every step rounds each stored moving population once; the second step
    # starts from a state carrying the first step's rounding
    assert rel_linf(phi1, rphi) <= (1e-5 if steps == 1 else 2 * u)
    assert np.abs(h1 - rh).max() <= steps * 15 * u * np.abs(rh).max() + 1e-5 * np.abs(rh).max()
    assert np.abs(g1 - rg).max() <= steps * q * u * np.abs(rg).max() + 1e-5 * np.abs(rg).max()


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_pair_matches_cell_form_on_a_step(lbm, prec):
    """From the same representable state the two fused variants store the same
    16-bit populations up to one unit of the format (they round the same FP32
    values, which differ in the last FP32 bits where the multiply-adds are fused
    differently)."""
    prob = W.Problem(66, 17, 11, wall=(1, 0, 1), q_hydro=27, rho_ratio=100.0, mu_ratio=30.0, sigma=1e-3, xi=3.0,
                     mobility=0.03, gravity=(1e-5, -2e-5, 3e-6), rho_ref=0.4, store_phi_ref=0.0)
    h, g, phi = W.random_state(prob, seed=11)
    out = {}
    for form in ("cell", "pair"):
        sim = lbm.Simulation.from_problem(prob, precision=prec, form=form)
        sim.set_state(h, g, phi)
        sim.step(1)
        out[form] = sim.get_state()
        sim.close()
    u = UNIT[prec]
    for a, b in zip(out["cell"], out["pair"]):
        assert np.abs(a - b).max() <= 2 * u * np.abs(b).max() + 1e-6 * np.abs(b).max()


def test_pair_static_droplet_200_steps(lbm, orc):
    """32^3 periodic droplet (D3Q15 + D3Q19, density ratio 1000), 200 steps, FP32:
    the same bounds as the one-cell form."""
    prob, phi0 = W.static_droplet()
    sim = lbm.Simulation.from_problem(prob, form="pair")
    sim.init_phase(phi0)
    m0 = sim.reduce()["mass"]
    sim.step(200)
    sim.synchronize()
    phi, u, p = (t.cpu().numpy() for t in sim.fields())
    m1 = sim.reduce()["mass"]
    rphi, ru, rp = orc.State(orc.make_problem(prob), phi0).run(200).fields()
    assert rel_linf(phi, rphi) <= TOL
    assert rel_linf(u, ru, 1e-6) <= TOL
    assert rel_linf(p, rp) <= TOL
    assert abs(m1 - m0) <= 1e-6 * abs(m0)


def test_pair_walled_bubble_200_steps(lbm, orc):
    """64^3 walled rising bubble, 200 steps, FP32 pair form: the bounds of
    test_gpu_walled (phi within 1e-5 off the heavy bulk, u and p within 1e-5)."""
    prob, phi0 = W.precision_bubble()
    sim = lbm.Simulation.from_problem(prob, form="pair")
    sim.init_phase(phi0)
    sim.step(200)
    sim.synchronize()
    phi, u, p = sim.fields(on_device=False)
    d = sim.reduce()
    rphi, ru, rp = orc.State(orc.make_problem(prob), phi0).run(200).fields()
    bubble = rphi < 0.999
    err = np.abs(phi.astype(np.float64) - rphi)
    assert err[bubble].max() <= TOL
    assert err.max() <= 2e-4
    assert rel_linf(u, ru, 1e-6) <= TOL
    assert rel_linf(p, rp) <= TOL
    ref = orc.diagnostics(prob, rphi, ru)
    assert abs(d["mass"] - ref["mass"]) <= 1e-6 * ref["mass"]
    assert abs(d["light_y"] - ref["light_y"]) <= 1e-4


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_pair_mass_kept_with_16bit_storage(lbm, prec):
    prob, phi0 = W.static_droplet()
    sim = lbm.Simulation.from_problem(prob, precision=prec, form="pair")
    sim.init_phase(phi0)
    m0 = sim.reduce()["mass"]
    sim.step(200)
    sim.synchronize()
    assert abs(sim.reduce()["mass"] - m0) <= 1e-6 * m0


def test_pair_split_steps_bitwise(lbm):
    prob, phi0 = W.static_droplet(n=20, radius=6.0, q_hydro=27)
    a = lbm.Simulation.from_problem(prob, precision="fp16", form="pair")
    a.init_phase(phi0)
    a.step(9)
    b = lbm.Simulation.from_problem(prob, precision="fp16", form="pair")
    b.init_phase(phi0)
    b.step(4)
    b.step(5)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
