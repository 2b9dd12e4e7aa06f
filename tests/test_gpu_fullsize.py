"""Parity at the benchmark's full size, in the benchmark's launch configuration.

The 512^3 roofline workload (D3Q15 + D3Q27, 400 bubbles) is advanced on the GPU
through the C ABI.  For sampled cells, the one-step update is recomputed by the
FP64 oracle: the new h, g and phi at a cell depend only on the state within
distance 2 (streaming from x - e_i, whose collision reads phi at x - e_i + e_j),
so the oracle steps a 5^3 periodic patch cut around the cell and its centre is
compared with the GPU.  Global properties (mass conservation, finiteness) are
checked on the whole field.
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


def patch(arr, z, y, x, r=2):
    """(..., 2r+1, 2r+1, 2r+1) periodic cut of a device tensor around (z, y, x), to numpy."""
    import torch

    nz, ny, nx = arr.shape[-3:]
    iz = torch.tensor([(z + d) % nz for d in range(-r, r + 1)], device=arr.device)
    iy = torch.tensor([(y + d) % ny for d in range(-r, r + 1)], device=arr.device)
    ix = torch.tensor([(x + d) % nx for d in range(-r, r + 1)], device=arr.device)
    out = arr.index_select(-3, iz).index_select(-2, iy).index_select(-1, ix)
    return out.double().cpu().numpy()


def wall_patch(arr, cell, prob, r=2):
    """(..., 5, 5, 5) cut around cell (z, y, x) of a walled or periodic box: along
    an axis whose walls lie within r of the cell, the cut starts (or ends) at the
    wall and the patch has walls on that axis (the patch's other face is more than
    r away from the cell); elsewhere a periodic cut centred on the cell.  Returns
    the cut, the cell's position in it and the patch's walls (x, y, z)."""
    import torch

    shape = arr.shape[-3:]
    walls_zyx = (prob.wall[2], prob.wall[1], prob.wall[0])
    idx, centre, pw = [], [], []
    for a in range(3):
        n, c, w = shape[a], cell[a], walls_zyx[a]
        if w and c < r:
            lo, walled = 0, 1
        elif w and c > n - 1 - r:
            lo, walled = n - (2 * r + 1), 1
        else:
            lo, walled = c - r, 0
        idx.append(torch.tensor([(lo + d) % n for d in range(2 * r + 1)], device=arr.device))
        centre.append(c - lo)
        pw.append(walled)
    out = arr.index_select(-3, idx[0]).index_select(-2, idx[1]).index_select(-1, idx[2])
    return out.double().cpu().numpy(), tuple(centre), (pw[2], pw[1], pw[0])


def check_sampled_step(lbm, orc, sim, prob, cells):
    """One GPU step from the current state vs the oracle on 5^3 patches (walled
    where the cell is within two cells of a walled face)."""
    h0, g0, phi0 = sim.get_state(on_device=True)
    sim.step(1)
    h1, g1, phi1 = sim.get_state(on_device=True)
    worst = 0.0
    for z, y, x in cells:
        hp, (cz, cy, cx), pw = wall_patch(h0, (z, y, x), prob)
        gp, _, _ = wall_patch(g0, (z, y, x), prob)
        fp, _, _ = wall_patch(phi0, (z, y, x), prob)
        sub = W.Problem(5, 5, 5, wall=pw, q_hydro=prob.q_hydro, rho_H=prob.rho_H, rho_ratio=prob.rho_ratio,
                        nu_H=prob.nu_H, mu_ratio=prob.mu_ratio, sigma=prob.sigma, xi=prob.xi,
                        mobility=prob.mobility, gravity=prob.gravity, rho_ref=prob.rho_ref, clamp_phi=prob.clamp_phi,
                        phase_mrt=prob.phase_mrt)
        p = orc.make_problem(sub)
        g_next, u = orc.hydro_step(p, gp, fp)
        h_next, phi_next = orc.phase_step(p, hp, fp, u)
        got_h = h1[:, z, y, x].double().cpu().numpy()
        got_g = g1[:, z, y, x].double().cpu().numpy()
        got_phi = float(phi1[z, y, x])
        rh, rg, rf = h_next[:, cz, cy, cx], g_next[:, cz, cy, cx], phi_next[cz, cy, cx]
        e_h = np.abs(got_h - rh).max() / max(np.abs(rh).max(), 1e-3)
        e_g = np.abs(got_g - rg).max() / max(np.abs(rg).max(), 1e-6)
        e_p = abs(got_phi - rf) / max(abs(rf), 1e-3)
        worst = max(worst, e_h, e_g, e_p)
        assert e_h <= TOL and e_g <= TOL and e_p <= TOL, (z, y, x, e_h, e_g, e_p)
    return worst


def test_roofline_512_sampled_one_step_parity(lbm, orc):
    import torch

    prob, phi0, bubbles = W.roofline()
    sim = lbm.Simulation.from_problem(prob)
    sim.init_phase(torch.from_numpy(phi0).cuda())
    rng = np.random.default_rng(6144)
    n = prob.nx
    cells = [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(48)]
    # cells on the interfaces of a few bubbles, and on the box faces (periodic wrap)
    for cx, cy, cz, r in bubbles[:16]:
        cells.append((int(cz) % n, int(cy) % n, int(cx + r) % n))
    cells += [(0, 0, 0), (n - 1, n - 1, n - 1), (0, n - 1, 5), (n - 1, 3, 0)]
    for warm in (0, 2):  # both in-place layouts of each lattice
        sim.step(warm)
        check_sampled_step(lbm, orc, sim, prob, cells)
    sim.synchronize()
    del sim
    torch.cuda.empty_cache()


def test_roofline_512_mass_and_finiteness(lbm):
    import torch

    prob, phi0, _ = W.roofline()
    sim = lbm.Simulation.from_problem(prob)
    sim.init_phase(torch.from_numpy(phi0).cuda())
    m0 = sim.reduce()["mass"]
    sim.step(50)
    sim.synchronize()
    d = sim.reduce()
    assert np.isfinite(list(d.values())).all()
    assert abs(d["mass"] - m0) <= 1e-6 * m0
    assert d["max_u"] < 0.1
    del sim
    torch.cuda.empty_cache()


@pytest.mark.parametrize("form,mrt", [("fused", 0), ("cell", 0), ("fused", 1), ("cell", 1)])
def test_beyond_32bit_offsets_sampled_parity(lbm, orc, form, mrt):
    """A box whose moving-plane offsets exceed 32 bits (26 N >= 2^32: 576 x 576 x 544,
    180 M cells) runs the fused step with 64-bit plane offsets (two cells per
    thread) or 64-bit plane pointers (one cell per thread), with the SRT and the
    MRT phase collision; sampled one-step parity in both in-place layouts, as for
    the 512^3 benchmark box."""
    import torch

    nx, ny, nz = 576, 576, 544
    assert 26 * nx * ny * nz >= 2 ** 32
    prob = W.Problem(nx, ny, nz, wall=(0, 0, 0), q_hydro=27, rho_ratio=100.0, sigma=1e-3, xi=4.0,
                     gravity=(0.0, -1e-6, 0.0), rho_ref=0.5, clamp_phi=1, phase_mrt=mrt)
    two_pi = 2.0 * np.pi
    x = torch.arange(nx, device="cuda", dtype=torch.float32) + 0.5
    y = torch.arange(ny, device="cuda", dtype=torch.float32) + 0.5
    z = torch.arange(nz, device="cuda", dtype=torch.float32) + 0.5
    phi0 = (0.5 + 0.45 * torch.sin(two_pi * x / nx)[None, None, :] * torch.sin(two_pi * 3 * y / ny)[None, :, None]
            * torch.cos(two_pi * 2 * z / nz)[:, None, None]).contiguous()
    sim = lbm.Simulation.from_problem(prob, form=form)
    sim.init_phase(phi0)
    rng = np.random.default_rng(576)
    cells = [(int(rng.integers(0, nz)), int(rng.integers(0, ny)), int(rng.integers(0, nx))) for _ in range(24)]
    cells += [(0, 0, 0), (nz - 1, ny - 1, nx - 1), (nz - 1, 0, nx - 1)]
    for warm in (0, 1):
        sim.step(warm)
        check_sampled_step(lbm, orc, sim, prob, cells)
    sim.synchronize()
    del sim
    torch.cuda.empty_cache()


def test_rising_bubble_walled_sampled_parity(lbm, orc):
    """The rising-bubble benchmark box (128 x 512 x 128, walls on every face,
    D3Q15 + D3Q27, D = 32, Eo 10, Mo 1e-3) after 40 steps: sampled one-step parity
    in both in-place layouts at random cells, on the bubble's interface, next to
    every face, along edges and in the corners (walled 5^3 patches there)."""
    import torch

    prob, phi0 = W.rising_bubble()
    sim = lbm.Simulation.from_problem(prob)
    sim.init_phase(torch.from_numpy(phi0).cuda())
    sim.step(40)
    rng = np.random.default_rng(128)
    nz, ny, nx = prob.shape
    cells = [(int(rng.integers(0, nz)), int(rng.integers(0, ny)), int(rng.integers(0, nx))) for _ in range(24)]
    cells += [(64, 64 + 16, 64), (64, 64 - 16, 64), (64 + 16, 64, 64), (64, 64, 64 - 16)]  # interface
    for d in (0, 1):
        cells += [(d, 200, 60), (nz - 1 - d, 200, 60), (70, d, 60), (70, ny - 1 - d, 60), (70, 200, d),
                  (70, 200, nx - 1 - d)]
    cells += [(0, 0, 0), (nz - 1, ny - 1, nx - 1), (0, ny - 1, nx - 1), (nz - 1, 0, 1), (1, 1, nx - 2), (0, 300, 0)]
    for warm in (0, 2):
        sim.step(warm)
        check_sampled_step(lbm, orc, sim, prob, cells)
    sim.synchronize()
    del sim
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_storage_formats_timing_box_sampled_parity(lbm, orc, prec):
    """The storage formats' timing box as the benchmark runs it (512^3, walls on
    every face, D = 32 at (256, 64, 256), 16-bit moving populations): after 10
    steps, one step at sampled cells (random, the bubble's interface, faces,
    edges, corners) against the oracle stepping walled / periodic 5^3 patches of
    the decoded state.  Each stored population rounds once (unit roundoff u of
    the format); the rest populations carry the others' rounding."""
    import torch

    unit = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}[prec]
    prob, phi0 = W.precision_timing(512)
    sim = lbm.Simulation.from_problem(prob, precision=prec)
    sim.init_phase(torch.from_numpy(phi0).cuda())
    sim.step(10)
    h0, g0, f0 = sim.get_state(on_device=True)
    sim.step(1)
    h1, g1, f1 = sim.get_state(on_device=True)
    rng = np.random.default_rng(512)
    n = 512
    cells = [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(16)]
    cells += [(256, 64 + 16, 256), (256, 64, 256 + 16), (256 - 16, 64, 256)]
    cells += [(0, 0, 0), (n - 1, n - 1, n - 1), (1, 300, n - 2), (n - 1, 0, 100), (200, n - 1, 0)]
    for z, y, x in cells:
        hp, (cz, cy, cx), pw = wall_patch(h0, (z, y, x), prob)
        gp, _, _ = wall_patch(g0, (z, y, x), prob)
        fp, _, _ = wall_patch(f0, (z, y, x), prob)
        sub = W.Problem(5, 5, 5, wall=pw, q_hydro=prob.q_hydro, rho_H=prob.rho_H, rho_ratio=prob.rho_ratio,
                        nu_H=prob.nu_H, mu_ratio=prob.mu_ratio, sigma=prob.sigma, xi=prob.xi,
                        mobility=prob.mobility, gravity=prob.gravity, rho_ref=prob.rho_ref, clamp_phi=prob.clamp_phi,
                        phase_mrt=prob.phase_mrt)
        p = orc.make_problem(sub)
        g_next, u = orc.hydro_step(p, gp, fp)
        h_next, phi_next = orc.phase_step(p, hp, fp, u)
        rh, rg, rf = h_next[:, cz, cy, cx], g_next[:, cz, cy, cx], phi_next[cz, cy, cx]
        got_h = h1[:, z, y, x].double().cpu().numpy()
        got_g = g1[:, z, y, x].double().cpu().numpy()
        # stored h_i - w_i phi_ref rounds once (phi_ref = 1): |stored| <= |h_i| + w_i
        assert abs(float(f1[z, y, x]) - rf) <= 1e-5 * max(abs(rf), 1e-2), (z, y, x)
        assert np.abs(got_h - rh).max() <= 15 * unit * (np.abs(rh).max() + 1.0) + 1e-5 * np.abs(rh).max(), (z, y, x)
        assert np.abs(got_g - rg).max() <= prob.q_hydro * unit * np.abs(rg).max() + 1e-5 * np.abs(rg).max() + 1e-9, (z, y, x)
    sim.synchronize()
    del sim
    torch.cuda.empty_cache()

