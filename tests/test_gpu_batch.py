"""Batched stepping (lbm_batch_*) through the C ABI.

A batch member runs the single-simulation step's code on its own cells; only
the assignment of tiles to thread blocks and the kernel around it differ.  The
first step is therefore bit-identical to a single run (every population of both
lattices and phi).  Later steps may differ in the last bit where the compiler
fuses a multiply and an add differently in the two kernels, and the flow
amplifies such differences like any rounding.  So after many steps each member
is held to the FP64 oracle: its phi, u and p are no further from the oracle
than the single-simulation path's (itself parity-tested), through plain
launches, CUDA-graph replay, every tile shape and table order the autotuner
visits, and a group boundary (more than 64 members per batch).  Two steps from
a random state are compared population by population with the oracle.
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


@pytest.fixture(scope="module")
def stream(lbm):
    import torch

    return torch.cuda.Stream()  # a non-default stream: the batch may use CUDA graphs


def _members(q):
    """Heterogeneous problems: several tiles and ragged tails, every wall
    combination kind, different physical parameters; a bubble or droplet each."""
    specs = [
        ((37, 29, 19), (0, 0, 0), dict(rho_ratio=100.0, mu_ratio=30.0, sigma=1e-3, xi=3.0, mobility=0.03,
                                       gravity=(1e-5, -2e-5, 3e-6), rho_ref=0.4), False),
        ((33, 17, 11), (1, 1, 1), dict(rho_ratio=1000.0, sigma=5e-4, xi=4.0, gravity=(0.0, -1e-5, 0.0),
                                       rho_ref=1.0, clamp_phi=1), False),
        ((64, 12, 10), (1, 0, 0), dict(rho_ratio=10.0, mu_ratio=5.0, nu_H=0.05, sigma=1e-4), True),
        ((5, 3, 2), (0, 1, 0), dict(rho_ratio=100.0, sigma=1e-3, xi=2.0), True),
        ((32, 8, 8), (0, 0, 1), dict(rho_ratio=1000.0, nu_H=0.02, mobility=0.05, gravity=(0.0, 0.0, 2e-6),
                                     rho_ref=1.0, clamp_phi=1), False),
    ]
    out = []
    for (nx, ny, nz), wall, kw, heavy in specs:
        prob = W.Problem(nx, ny, nz, wall=wall, q_hydro=q, **kw)
        r = max(1.0, min(nx, ny, nz) / 3.0)
        phi0 = W.sphere_phi(prob, (nx / 2, ny / 2, nz / 2), r, heavy_inside=heavy).astype(np.float32)
        out.append((prob, phi0))
    return out


def _alone(lbm, prob, phi0, steps, what="state"):
    """The same problem stepped alone by the one-cell fused step, whose tile body
    the batched kernel shares."""
    sim = lbm.Simulation.from_problem(prob, form="cell")
    sim.init_phase(phi0)
    sim.step(steps)
    sim.synchronize()
    out = sim.get_state() if what == "state" else _fields(sim)
    sim.close()
    return out


def _fields(sim):
    return [t.cpu().numpy().astype(np.float64) for t in sim.fields()]


def _assert_same(a, b):
    for x, y, name in zip(a, b, ("h", "g", "phi")):
        assert np.isfinite(y).all()
        assert np.array_equal(x, y), f"{name}: max diff {np.abs(x - y).max()}"


def _assert_as_close_as_single(orc, lbm, member, prob, phi0, steps):
    """phi, u, p of a batch member are no further from the FP64 oracle than those
    of the same problem stepped alone: within 3 times the single run's distance
    (two trajectories that differ by rounding scatter about the oracle alike),
    plus 1e-5 of the field's scale (the parity tolerance; it covers a single run
    that happens to land very close)."""
    b = _fields(member)
    s = _alone(lbm, prob, phi0, steps, what="fields")
    o = orc.State(orc.make_problem(prob), phi0).run(steps).fields()
    for name, bf, sf, of, floor in zip(("phi", "u", "p"), b, s, o, (0.0, 1e-6, 1e-9)):
        assert np.isfinite(bf).all()
        eb, es = np.abs(bf - of).max(), np.abs(sf - of).max()
        assert eb <= 3.0 * es + TOL * max(np.abs(of).max(), floor), f"{name}: batch {eb:.3e} single {es:.3e}"


@pytest.mark.parametrize("q", [19, 27])
def test_first_step_bit_identical(lbm, stream, q):
    members = _members(q)
    batch = lbm.Batch.from_problems([p for p, _ in members], stream=stream)
    for m, (_, phi0) in zip(batch.members, members):
        m.init_phase(phi0)
    batch.step(1)
    batch.synchronize()
    for m, (prob, phi0) in zip(batch.members, members):
        _assert_same(m.get_state(), _alone(lbm, prob, phi0, 1))
    batch.close()


@pytest.mark.parametrize("q", [19, 27])
def test_members_match_single_runs(lbm, orc, stream, q):
    members = _members(q)
    batch = lbm.Batch.from_problems([p for p, _ in members], stream=stream)
    for m, (_, phi0) in zip(batch.members, members):
        m.init_phase(phi0)
    batch.step(3)   # plain launches
    batch.step(16)  # one graph replay
    batch.step(21)  # a graph replay and 5 plain launches
    batch.synchronize()
    assert batch.steps_done() == 40
    for m, (prob, phi0) in zip(batch.members, members):
        assert m.steps_done() == 40
        _assert_as_close_as_single(orc, lbm, m, prob, phi0, 40)
    batch.close()


def test_tuner_visits_every_candidate(lbm, orc, stream):
    """The tuner's trial steps are real steps through the one-cell tile shapes x
    2 table orders; these members (some nx odd) have neither the two-cell tiles
    nor the TMA staging, so those 10 candidates are skipped.  The members must still match single runs afterwards."""
    members = _members(27)
    batch = lbm.Batch.from_problems([p for p, _ in members], stream=stream)
    for m, (_, phi0) in zip(batch.members, members):
        m.init_phase(phi0)
    shape, order, halo, ms = batch.tune(trial_steps=2)
    assert shape in lbm.BATCH_SHAPES and order in lbm.BATCH_ORDERS and halo == "loads"
    # odd nx: no two-cell tiles (candidates 6, 7) and no TMA staging (8..15)
    assert ms.shape == (16,) and np.all(ms[:6] > 0) and np.all(ms[6:] == -1.0)
    assert batch.steps_done() == 6 * 3
    with pytest.raises(lbm.LBMError) as e:
        batch.configure((4, 2), "member", "tma")
    assert e.value.status == lbm.LBM_ERR_STATE
    batch.step(17)  # the chosen candidate, graph and plain
    batch.synchronize()
    for m, (prob, phi0) in zip(batch.members, members):
        _assert_as_close_as_single(orc, lbm, m, prob, phi0, 6 * 3 + 17)
    batch.close()


def test_refused_configuration_keeps_the_current_one(lbm, orc, stream):
    """A configuration the batch refuses (TMA staging for members whose nx is not
    a multiple of 4) leaves the one in use untouched: the tile table still
    matches the kernel that the next step launches."""
    members = _members(27)
    batch = lbm.Batch.from_problems([p for p, _ in members], stream=stream)
    for m, (_, phi0) in zip(batch.members, members):
        m.init_phase(phi0)
    batch.configure((2, 4), "round_robin", "loads")
    with pytest.raises(lbm.LBMError) as e:
        batch.configure((4, 2), "member", "tma")
    assert e.value.status == lbm.LBM_ERR_STATE
    batch.step(3)
    batch.step(16)
    batch.synchronize()
    for m, (prob, phi0) in zip(batch.members, members):
        _assert_as_close_as_single(orc, lbm, m, prob, phi0, 19)
    batch.close()


def _tma_members(q):
    """Members whose rows suit the TMA staging (nx a multiple of 4): several x
    tiles and a ragged x tail, ragged y / z tails, walled and periodic faces on
    every axis (periodic-face tiles fall back to per-thread loads)."""
    specs = [
        ((36, 29, 19), (1, 1, 1), dict(rho_ratio=100.0, mu_ratio=30.0, sigma=1e-3, xi=3.0, mobility=0.03,
                                       gravity=(1e-5, -2e-5, 3e-6), rho_ref=0.4), False),
        ((96, 17, 11), (0, 0, 0), dict(rho_ratio=1000.0, sigma=5e-4, xi=4.0, gravity=(0.0, -1e-5, 0.0),
                                       rho_ref=1.0, clamp_phi=1), False),
        ((64, 13, 10), (1, 0, 1), dict(rho_ratio=10.0, mu_ratio=5.0, nu_H=0.05, sigma=1e-4), True),
        ((8, 9, 7), (0, 1, 0), dict(rho_ratio=10.0, sigma=1e-4, xi=3.0), True),
        ((100, 12, 9), (1, 1, 0), dict(rho_ratio=1000.0, nu_H=0.02, mobility=0.05, gravity=(0.0, 0.0, 2e-6),
                                       rho_ref=1.0, clamp_phi=1), False),
    ]
    out = []
    for (nx, ny, nz), wall, kw, heavy in specs:
        prob = W.Problem(nx, ny, nz, wall=wall, q_hydro=q, **kw)
        r = max(1.0, min(nx, ny, nz) / 3.0)
        phi0 = W.sphere_phi(prob, (nx / 2, ny / 2, nz / 2), r, heavy_inside=heavy).astype(np.float32)
        out.append((prob, phi0))
    return out


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("shape", [(4, 2), (8, 1), (2, 4)])
def test_tma_halo_staging(lbm, orc, stream, q, shape):
    """The TMA-staged phi tile feeds the same stencil values as per-thread loads:
    one step from a random state agrees with the loads' step to FP32 rounding (the
    two kernels may contract multiply-adds differently) and with the FP64 oracle;
    after plain and graph-replayed steps every member is as close to the oracle
    as a single run."""
    members = _tma_members(q)
    states = [W.random_state(p, seed=31 + k) for k, (p, _) in enumerate(members)]
    got = {}
    for halo in ("loads", "tma"):
        batch = lbm.Batch.from_problems([p for p, _ in members], stream=stream)
        batch.configure(shape, "member", halo)
        for m, st in zip(batch.members, states):
            m.set_state(*st)
        batch.step(1)
        batch.synchronize()
        got[halo] = [m.get_state() for m in batch.members]
        batch.close()
    for (prob, _), st, a, b in zip(members, states, got["loads"], got["tma"]):
        h, g, phi = st
        op = orc.make_problem(prob)
        g1, u = orc.hydro_step(op, g.astype(np.float64), phi.astype(np.float64))
        h1, phi1 = orc.phase_step(op, h.astype(np.float64), phi.astype(np.float64), u)
        for x, y, ref in zip(a, b, (h1, g1, phi1)):
            scale = np.abs(ref).max()
            assert np.abs(x - y).max() <= 1e-6 * scale
            assert np.abs(y - ref).max() <= TOL * scale
    batch = lbm.Batch.from_problems([p for p, _ in members], stream=stream)
    batch.configure(shape, "round_robin", "tma")
    for m, (_, phi0) in zip(batch.members, members):
        m.init_phase(phi0)
    batch.step(3)
    batch.step(16)
    batch.synchronize()
    for m, (prob, phi0) in zip(batch.members, members):
        _assert_as_close_as_single(orc, lbm, m, prob, phi0, 19)
    batch.close()


def test_tuner_with_tma_candidates(lbm, orc, stream):
    """With TMA-capable members (nx multiples of 4) the tuner times 14 candidates:
    every one but the two-cell tiles with TMA staging."""
    members = _tma_members(27)
    batch = lbm.Batch.from_problems([p for p, _ in members], stream=stream)
    for m, (_, phi0) in zip(batch.members, members):
        m.init_phase(phi0)
    shape, order, halo, ms = batch.tune(trial_steps=2)
    assert ms.shape == (16,) and np.all(ms[:14] > 0) and np.all(ms[14:] == -1.0)
    assert halo in lbm.BATCH_HALOS
    assert batch.steps_done() == 14 * 3
    batch.step(5)
    batch.synchronize()
    for m, (prob, phi0) in zip(batch.members, members):
        _assert_as_close_as_single(orc, lbm, m, prob, phi0, 14 * 3 + 5)
    batch.close()


@pytest.mark.parametrize("q", [19, 27])
def test_two_cell_tiles(lbm, orc, stream, q):
    """The two-cells-per-thread tiles (32 x 4 x 2 cells) on members with nx even,
    walled and periodic faces and ragged tails: two steps from a random state
    against the FP64 oracle population by population, then plain and
    graph-replayed steps as close to the oracle as single runs; a batch with an
    odd nx refuses the shape."""
    members = _tma_members(q)
    states = [W.random_state(p, seed=51 + k) for k, (p, _) in enumerate(members)]
    batch = lbm.Batch.from_problems([p for p, _ in members], stream=stream)
    batch.configure("pair", "round_robin", "loads")
    for m, st in zip(batch.members, states):
        m.set_state(*st)
    batch.step(2)
    batch.synchronize()
    for m, (prob, _), (h, g, phi) in zip(batch.members, members, states):
        op = orc.make_problem(prob)
        for _ in range(2):
            g, u = orc.hydro_step(op, g.astype(np.float64), phi.astype(np.float64))
            h, phi = orc.phase_step(op, h.astype(np.float64), phi.astype(np.float64), u)
        for a, b in zip(m.get_state(), (h, g, phi)):
            assert np.abs(a - b).max() <= TOL * np.abs(b).max()
    batch.close()
    batch = lbm.Batch.from_problems([p for p, _ in members], stream=stream)
    batch.configure("pair", "member", "loads")
    for m, (_, phi0) in zip(batch.members, members):
        m.init_phase(phi0)
    batch.step(3)
    batch.step(16)
    batch.synchronize()
    for m, (prob, phi0) in zip(batch.members, members):
        _assert_as_close_as_single(orc, lbm, m, prob, phi0, 19)
    batch.close()
    odd = _members(q)
    batch = lbm.Batch.from_problems([p for p, _ in odd], stream=stream)
    with pytest.raises(lbm.LBMError) as e:
        batch.configure("pair", "member", "loads")
    assert e.value.status == lbm.LBM_ERR_STATE
    batch.close()


def test_group_boundary(lbm, orc, stream):
    """70 members: two launches per step (64 + 6 members)."""
    rng = np.random.default_rng(70)
    members = []
    for i in range(70):
        nx, ny, nz = int(rng.integers(1, 40)), int(rng.integers(1, 12)), int(rng.integers(1, 6))
        wall = tuple(int(v) for v in rng.integers(0, 2, size=3))
        prob = W.Problem(nx, ny, nz, wall=wall, q_hydro=27, rho_ratio=float(rng.choice([10.0, 100.0])),
                         sigma=1e-3, xi=2.0, gravity=(0.0, -1e-5, 0.0), rho_ref=1.0, clamp_phi=1)
        phi0 = W.random_smooth_field(prob.shape, rng).astype(np.float32)
        members.append((prob, phi0))
    batch = lbm.Batch.from_problems([p for p, _ in members], stream=stream)
    for m, (_, phi0) in zip(batch.members, members):
        m.init_phase(phi0)
    batch.step(17)
    batch.synchronize()
    for m, (prob, phi0) in zip(batch.members, members):
        _assert_as_close_as_single(orc, lbm, m, prob, phi0, 17)
    batch.close()


def test_member_two_steps_against_oracle(lbm, orc, stream):
    """Both in-place layouts of a batch member against the FP64 oracle, from a
    random state (every population compared)."""
    probs = [W.Problem(37, 29, 19, wall=(1, 0, 1), q_hydro=27, rho_ratio=100.0, mu_ratio=30.0, sigma=1e-3,
                       xi=3.0, mobility=0.03, gravity=(1e-5, -2e-5, 3e-6), rho_ref=0.4),
             W.Problem(9, 40, 3, wall=(0, 1, 0), q_hydro=27)]
    batch = lbm.Batch.from_problems(probs, stream=stream)
    states = [W.random_state(p, seed=11 + k) for k, p in enumerate(probs)]
    for m, st in zip(batch.members, states):
        m.set_state(*st)
    batch.step(2)
    batch.synchronize()
    for m, p, (h, g, phi) in zip(batch.members, probs, states):
        op = orc.make_problem(p)
        for _ in range(2):
            g, u = orc.hydro_step(op, g.astype(np.float64), phi.astype(np.float64))
            h, phi = orc.phase_step(op, h.astype(np.float64), phi.astype(np.float64), u)
        h2, g2, phi2 = m.get_state()
        for a, b in ((phi2, phi), (h2, h), (g2, g)):
            assert np.abs(a - b).max() <= TOL * np.abs(b).max()
    batch.close()


def test_batched_workload_members(lbm, orc, stream):
    """The batched rising-bubble recipe (first 6 draws) over two graph replays:
    mass kept; the members up to 48 x 96 x 48 cells as close to the oracle as
    single runs."""
    draws = W.batched(count=6)
    batch = lbm.Batch.from_problems([p for p, _, _ in draws], stream=stream)
    for m, (_, phi0, _) in zip(batch.members, draws):
        m.init_phase(phi0)
    m0 = [m.reduce()["mass"] for m in batch.members]
    batch.step(32)
    batch.synchronize()
    for k, (m, (prob, phi0, _)) in enumerate(zip(batch.members, draws)):
        assert abs(m.reduce()["mass"] - m0[k]) <= 1e-6 * m0[k]
        if prob.ncells <= 48 * 96 * 48:
            _assert_as_close_as_single(orc, lbm, m, prob, phi0, 32)
    batch.close()


def test_batch_errors(lbm, stream):
    a = W.Problem(8, 8, 8, q_hydro=27)
    b = W.Problem(8, 8, 8, q_hydro=19)
    with pytest.raises(lbm.LBMError) as e:
        lbm.Batch.from_problems([a, b], stream=stream)
    assert e.value.status == lbm.LBM_ERR_ARG
    c = W.Problem(8, 8, 8, q_hydro=27, precision="fp16")
    with pytest.raises(lbm.LBMError) as e:
        lbm.Batch.from_problems([a, c], stream=stream)
    assert e.value.status == lbm.LBM_ERR_ARG
    batch = lbm.Batch.from_problems([a, a], stream=stream)
    with pytest.raises(lbm.LBMError) as e:
        batch.step(1)  # no state yet
    assert e.value.status == lbm.LBM_ERR_STATE
    phi0 = W.sphere_phi(a, (4, 4, 4), 2.5, heavy_inside=True).astype(np.float32)
    for m in batch.members:
        m.init_phase(phi0)
    batch.members[0].step(1)  # out of lockstep
    with pytest.raises(lbm.LBMError) as e:
        batch.step(1)
    assert e.value.status == lbm.LBM_ERR_STATE
    batch.members[1].step(1)
    batch.step(2)
    batch.synchronize()
    _assert_same(batch.members[0].get_state(), batch.members[1].get_state())
    batch.close()
