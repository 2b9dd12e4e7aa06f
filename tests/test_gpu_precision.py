"""Reduced-precision population storage (FP16, BF16; FP32 arithmetic) against the
FP64 oracle.

Storage: rest populations FP32; moving h_i as h_i - w_i ref, moving g_i as
g_i * scale, in 16 bits.  Bounds derive from the formats' unit roundoff u
(FP16 2^-11, BF16 2^-8): a stored moving population is off by at most u times
its stored magnitude, and the FP32 rest population absorbs the rounding of the
others, so phi (and p*) stay exact to FP32 rounding.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

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


def _stored(orc, h, ref):
    """Magnitudes the 16-bit formats hold for h (h_i - w_i ref)."""
    _, w, _ = orc.lattice(15)
    return np.abs(h - w[:, None, None, None] * ref)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_state_roundtrip_rounds_once(lbm, orc, prec):
    prob = W.Problem(13, 7, 5, wall=(1, 0, 1), q_hydro=27, store_phi_ref=1.0)
    h, g, phi = W.random_state(prob, seed=3)
    sim = lbm.Simulation.from_problem(prob, precision=prec)
    sim.set_state(h, g, phi)
    h1, g1, phi1 = sim.get_state()
    u = UNIT[prec]
    assert np.array_equal(phi1, phi)
    assert np.array_equal(h1[0], h[0]) and np.array_equal(g1[0], g[0])  # rest populations in FP32
    # relative rounding u for normal numbers, half the smallest subnormal step
    # (2^-25 for FP16) near zero, plus the FP32 rounding of w_i ref + q on decode
    sub = 2.0 ** -25 if prec == "fp16" else 0.0
    assert np.all(np.abs(h1[1:] - h[1:]) <= u * _stored(orc, h, 1.0)[1:] * 1.0001 + sub + 1e-8)
    assert np.all(np.abs(g1[1:] - g[1:]) <= u * np.abs(g[1:]) * 1.0001 + sub / 4096 + 1e-12)
    sim.set_state(h1, g1, phi1)
    for a, b in zip(sim.get_state(), (h1, g1, phi1)):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("nx,ny,nz,wall,q", [(37, 29, 19, (0, 0, 0), 19), (33, 17, 11, (1, 1, 1), 27)])
def test_one_step_parity(lbm, orc, prec, nx, ny, nz, wall, q):
    prob = W.Problem(nx, ny, nz, wall=wall, q_hydro=q, rho_ratio=100.0, mu_ratio=30.0, sigma=1e-3, xi=3.0,
                     mobility=0.03, gravity=(1e-5, -2e-5, 3e-6), rho_ref=0.4, store_phi_ref=0.0)
    h, g, phi = W.random_state(prob, seed=nx + ny + nz)
    sim = lbm.Simulation.from_problem(prob, precision=prec)
    sim.set_state(h, g, phi)
    h0, g0, phi0 = sim.get_state()  # the representable state the step starts from
    sim.step(1)
    sim.synchronize()
    h1, g1, phi1 = sim.get_state()
    p = orc.make_problem(prob)
    rg, u = orc.hydro_step(p, g0.astype(np.float64), phi0.astype(np.float64))
    rh, rphi = orc.phase_step(p, h0.astype(np.float64), phi0.astype(np.float64), u)
    uu = UNIT[prec]
    assert rel_linf(phi1, rphi) <= 1e-5
    # each output population rounds once; the rest population carries the others' rounding
    assert np.abs(h1 - rh).max() <= 15 * uu * np.abs(rh).max() + 1e-5 * np.abs(rh).max()
    assert np.abs(g1 - rg).max() <= q * uu * np.abs(rg).max() + 1e-5 * np.abs(rg).max()


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_mass_kept_with_16bit_storage(lbm, prec):
    prob, phi0 = W.static_droplet()
    sim = lbm.Simulation.from_problem(prob, precision=prec)
    sim.init_phase(phi0)
    m0 = sim.reduce()["mass"]
    sim.step(200)
    sim.synchronize()
    assert abs(sim.reduce()["mass"] - m0) <= 1e-6 * m0


def _rise(phi, u):
    lf = 1.0 - phi
    return float((u[1] * lf).sum() / lf.sum())


def test_precision_bubble_errors(lbm, orc):
    """64^3 walled rising bubble (D = 16, Eo 10, Mo 1e-3, t_ref 1000), 1000 steps:
    phi L-infinity, rise velocity and mass drift of each storage format against
    the FP64 oracle."""
    prob, phi0 = W.precision_bubble()
    steps = 1000
    ref = orc.State(orc.make_problem(prob), phi0).run(steps)
    rphi, ru, _ = ref.fields()
    r_rise = _rise(rphi, ru)
    m_ref = rphi.sum()
    errs = {}
    for prec in ("fp32", "fp16", "bf16"):
        sim = lbm.Simulation.from_problem(prob, precision=prec)
        sim.init_phase(phi0)
        sim.step(steps)
        sim.synchronize()
        phi, u, _ = (t.cpu().numpy().astype(np.float64) for t in sim.fields())
        errs[prec] = dict(phi_linf=float(np.abs(phi - rphi).max()),
                          rise_rel=abs(_rise(phi, u) - r_rise) / abs(r_rise),
                          mass_drift=abs(phi.sum() - m_ref) / m_ref)
        sim.close()
    print("precision errors vs FP64 oracle:", errs, "rise velocity", r_rise)
    # stated accuracy (64^3, 1000 steps; measured on a GB300: FP32 phi 5.6e-4,
    # rise 3.3e-6; FP16 4.2e-4, 1.3e-4; BF16 2.7e-3, 4.5e-3 -- the start from rest
    # amplifies rounding, so FP32 and FP16 are close in phi)
    assert errs["fp32"]["phi_linf"] <= 2e-3 and errs["fp32"]["rise_rel"] <= 1e-4
    assert errs["fp16"]["phi_linf"] <= 2e-3 and errs["fp16"]["rise_rel"] <= 1e-3
    assert errs["bf16"]["phi_linf"] <= 1e-2 and errs["bf16"]["rise_rel"] <= 2e-2
    for e in errs.values():
        assert e["mass_drift"] <= 1e-6
