"""The exchange sets of the sharded form (a z-slab per GPU, Section 4.2's
ghost-layer communication), checked on CPU with the oracle and two gloo ranks.

Only one GPU takes part in any run of this build, so the sharded data path
itself is not built; this test checks that the data a slab needs from its
neighbours per time step is exactly what the design sends:
  * before the phase step k: the neighbour's boundary layer of phi^{k-1}
    (the stencils of the normal and of the hydro forces reach one cell across
    the face);
  * after it: the h populations that left the neighbour's slab through the
    shared face (e_z pointing across it: 5 of the D3Q15 directions);
  * before the hydro step: the boundary layer of phi^k;
  * after it: the g populations that crossed the face (9 of the D3Q27
    directions).
Each rank steps its slab padded with one ghost layer per face (the oracle's
whole-box steps on the padded box; ghost cells carry zeros and their results
are discarded), sends what its boundary cells pushed into the ghost layers and
writes what it receives into its first and last layers.  After several steps
of a random state (walls on x, periodic y, and z periodic across the two
slabs) the slabs put together equal a whole-box oracle run bit for bit.
"""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


WORKER = r"""
import dataclasses, json, os, sys
import numpy as np
sys.path.insert(0, {root!r})
import torch
import torch.distributed as dist
import oracle
import workloads as W

rank = int(os.environ["RANK"]); world = int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo")
oracle.set_threads(1)
prob = W.Problem({nx}, {ny}, {nz}, wall=(1, 0, 0), q_hydro={q}, rho_ratio=100.0, mu_ratio=30.0, sigma=1e-3,
                 xi=3.0, mobility=0.03, gravity=(1e-5, -2e-5, 3e-6), rho_ref=0.4)
h, g, phi = (a.astype(np.float64) for a in W.random_state(prob, seed=7))
u = np.random.default_rng(8).normal(0.0, 1e-3, size=(3,) + phi.shape)
nzl = prob.nz // world
z0 = rank * nzl
up, down = (rank + 1) % world, (rank - 1) % world
slab = oracle.make_problem(dataclasses.replace(prob, nz=nzl + 2))

def padded(a):
    # slab [z0, z0 + nzl) with one ghost layer per face (zeros)
    out = np.zeros(a.shape[:-3] + (nzl + 2,) + a.shape[-2:])
    out[..., 1:-1, :, :] = a[..., z0:z0 + nzl, :, :]
    return out

def swap(send_up, send_down):
    # send_up goes to the slab above (its lower ghost), send_down to the one below;
    # tags keep the two directions apart when both neighbours are the same rank
    from_below = torch.empty(send_up.shape, dtype=torch.float64)
    from_above = torch.empty(send_down.shape, dtype=torch.float64)
    ops = [dist.P2POp(dist.isend, torch.from_numpy(np.ascontiguousarray(send_up)), up, tag=0),
           dist.P2POp(dist.irecv, from_below, down, tag=0),
           dist.P2POp(dist.isend, torch.from_numpy(np.ascontiguousarray(send_down)), down, tag=1),
           dist.P2POp(dist.irecv, from_above, up, tag=1)]
    for r in dist.batch_isend_irecv(ops):
        r.wait()
    return from_below.numpy(), from_above.numpy()

def fill_phi_ghosts(f):
    below, above = swap(f[-2], f[1])
    f[0], f[-1] = below, above

def crosses(ei):
    # cells (y, x) of a layer whose population e_i comes from the neighbour's
    # slab: its source (x - e_x, y - e_y) must not lie beyond a walled face (there
    # the cell's own population bounced back, and nothing crosses the face)
    xs, ys = np.arange(prob.nx) - ei[0], np.arange(prob.ny) - ei[1]
    mx = (xs >= 0) & (xs < prob.nx) if prob.wall[0] else np.ones(prob.nx, bool)
    my = (ys >= 0) & (ys < prob.ny) if prob.wall[1] else np.ones(prob.ny, bool)
    return my[:, None] & mx[None, :]

def exchange_populations(f, q):
    # what the boundary cells pushed into the ghost layers goes to the neighbour,
    # which writes it into its first / last layer (same x, y) where it crossed the face
    e = oracle.lattice(q)[0]
    zp, zn = np.nonzero(e[:, 2] > 0)[0], np.nonzero(e[:, 2] < 0)[0]
    below, above = swap(f[zp, -1], f[zn, 0])
    crossing = 0
    for k, i in enumerate(zp):
        m = crosses(e[i])
        f[i, 1][m] = below[k][m]
        crossing += int(m.sum())
    for k, i in enumerate(zn):
        m = crosses(e[i])
        f[i, -2][m] = above[k][m]
    f[:, 0] = 0.0
    f[:, -1] = 0.0
    return len(zp), crossing

hp, gp, phi_prev, up_ = padded(h), padded(g), padded(phi), padded(u)
sent = set()
for k in range({steps}):
    fill_phi_ghosts(phi_prev)
    hp, phi_now = oracle.phase_step(slab, hp, phi_prev, up_)
    sent.add(("h",) + exchange_populations(hp, 15))
    fill_phi_ghosts(phi_now)
    gp, up_ = oracle.hydro_step(slab, gp, phi_now)
    sent.add(("g",) + exchange_populations(gp, {q}))
    phi_prev = phi_now
    phi_prev[0] = phi_prev[-1] = 0.0
    up_[:, 0] = 0.0
    up_[:, -1] = 0.0

parts = [hp[:, 1:-1], gp[:, 1:-1], phi_prev[1:-1], up_[:, 1:-1]]
gathered = []
for a in parts:
    t = torch.from_numpy(np.ascontiguousarray(a))
    lst = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(lst, t)
    gathered.append(np.concatenate([x.numpy() for x in lst], axis=-3))
if rank == 0:
    ref = oracle.State(oracle.make_problem(prob), phi)
    ref.h[...] = h
    ref.g[...] = g
    ref.phi_prev[...] = phi
    ref.u_prev[...] = u
    ref.run({steps})
    names = ("h", "g", "phi", "u")
    same = {{n: bool(np.array_equal(a, b)) for n, a, b in
             zip(names, gathered, (ref.h, ref.g, ref.phi_prev, ref.u_prev))}}
    diff = {{n: float(np.abs(a - b).max()) for n, a, b in
             zip(names, gathered, (ref.h, ref.g, ref.phi_prev, ref.u_prev))}}
    print("RESULT " + json.dumps({{"same": same, "diff": diff, "sent": sorted(sent)}}), flush=True)
dist.destroy_process_group()
"""


@pytest.mark.parametrize("q", [27, 19])
def test_two_slabs_with_designed_exchange_match_whole_box(tmp_path, q):
    import oracle

    oracle.build()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "worker.py"
    script.write_text(WORKER.format(root=root, nx=9, ny=6, nz=8, q=q, steps=6))
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                   LOCAL_RANK=str(rank), OMP_NUM_THREADS="1")
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err
        outs.append(out)
    import json

    res = json.loads([l for l in outs[0].splitlines() if l.startswith("RESULT ")][0][len("RESULT "):])
    assert all(res["same"].values()), res
    # the exchanged sets per face: 5 of the D3Q15 directions, 9 of D3Q27 or 5 of D3Q19;
    # with walls on x (9 cells) and y periodic (6 cells), a direction with e_x != 0
    # crosses at 8 x 6 cells of the layer, one with e_x = 0 at 9 x 6
    e15 = oracle.lattice(15)[0]
    eg = oracle.lattice(q)[0]
    cells = lambda e: sum(6 * (8 if v[0] else 9) for v in e if v[2] > 0)
    assert sorted(map(tuple, res["sent"])) == [("g", 9 if q == 27 else 5, cells(eg)), ("h", 5, cells(e15))]
