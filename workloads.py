"""Seeded synthetic inputs for the conservative Allen-Cahn multiphase LBM.

This module holds only problem statements and initial phase fields: box sizes,
boundary types, physical parameters (densities, viscosities, surface tension,
interface width, mobility, gravity) and the initial phi0 built from the
equilibrium interface profile phi = 1/2 +- 1/2 tanh(2 d / xi) of Section 3.1
(d = signed distance to the interface).  It contains none of the lattice
Boltzmann arithmetic; both the CUDA library and the oracle receive the same
float32 phi0 from here.

Workloads (cell centres at i + 1/2, y is "up"):

* ``static_droplet``   32^3 periodic, D3Q15 + D3Q19, heavy droplet R = 8 at the
  centre, rho_H/rho_L = 1000, mu ratio 100, nu_H = 0.01, sigma = 1e-4, xi = 5,
  M = 0.02, no gravity.
* ``rising_bubble``    128 x 512 x 128, walls on every face, D3Q15 + D3Q27,
  bubble D = 32 at (64, 64, 64); Eo = 10, Mo = 1e-3, t_ref = sqrt(D/g) = 2000
  steps, M = 0.04 (Section 6.1 groups Re_Gr, Eo, t_ref).
* ``roofline``         512^3 triply periodic, D3Q15 + D3Q27, 400 non-overlapping
  bubbles with D ~ U[16, 32] placed by rejection sampling from
  ``numpy.random.default_rng(6144)``; gravity with Eo = 10 at D = 24;
  buoyancy reference = mean density (periodic gravity axis).
* ``precision_bubble`` 64^3 walled rising bubble, D = 16 at (32, 16, 32),
  Eo = 10, Mo = 1e-3, t_ref = 1000 (the storage formats' error case).
* ``precision_timing`` 512^3 walled rising bubble, D = 32 at (256, 64, 256),
  the rising-bubble parameters (the storage formats' timing case).
* ``batched``          64 walled rising bubbles of four box sizes, seeded draws of
  density ratio and Eo (batched stepping).
* ``roofline2d``       8192 x 16384 x 1 periodic, D2Q9 + D2Q9, light circles on a
  square lattice, the roofline physics (the two-dimensional pair).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Sequence

import numpy as np

SEED = 6144


@dataclasses.dataclass
class Problem:
    """Box, lattice choice and the physical parameters of Section 3."""

    nx: int
    ny: int
    nz: int
    wall: tuple = (0, 0, 0)  # 0 = periodic axis, 1 = no-slip walls on both faces
    q_hydro: int = 27
    q_phase: int = 15  # phase-field lattice: 15 (the benchmarked pair), 19, 27; 9 with q_hydro 9 (2-D)
    rho_H: float = 1.0
    rho_ratio: float = 1000.0
    nu_H: float = 0.01
    mu_ratio: float = 100.0
    sigma: float = 1e-4
    xi: float = 5.0
    mobility: float = 0.02
    gravity: tuple = (0.0, 0.0, 0.0)
    rho_ref: float = 1.0
    clamp_phi: int = 0  # 1: phi clamped to [0, 1] inside rho and tau
    phase_mrt: int = 0  # 1: MRT phase collision of Section 3.1 (0: SRT, the benchmarked form)
    unfused: int = 0  # 1: run the unfused baseline (Algorithm 1's passes) instead of the fused step
    precision: str = "fp32"  # population storage: "fp32", "fp16", "bf16"
    store_phi_ref: float = 0.0  # 16-bit storage keeps h_i - w_i store_phi_ref (1: mostly heavy fluid)

    @property
    def rho_L(self) -> float:
        return self.rho_H / self.rho_ratio

    @property
    def nu_L(self) -> float:
        # mu_H / mu_L = mu_ratio with mu = rho nu
        return self.nu_H * self.rho_H / (self.mu_ratio * self.rho_L)

    @property
    def shape(self) -> tuple:
        """Array shape of a scalar field, (nz, ny, nx): x is the fastest index."""
        return (self.nz, self.ny, self.nx)

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz


# ---------------------------------------------------------------------------
# phase-field geometry


def _axis_delta(coord: np.ndarray, centre: float, n: int, periodic: bool) -> np.ndarray:
    d = coord - centre
    if periodic:
        d = d - n * np.round(d / n)
    return d


def sphere_phi(prob: Problem, centre: Sequence[float], radius: float, heavy_inside: bool) -> np.ndarray:
    """phi0 of one sphere (float64, shape (nz, ny, nx)); minimum image on periodic axes."""
    z, y, x = np.meshgrid(
        np.arange(prob.nz) + 0.5, np.arange(prob.ny) + 0.5, np.arange(prob.nx) + 0.5, indexing="ij"
    )
    dx = _axis_delta(x, centre[0], prob.nx, not prob.wall[0])
    dy = _axis_delta(y, centre[1], prob.ny, not prob.wall[1])
    dz = _axis_delta(z, centre[2], prob.nz, not prob.wall[2])
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    s = 2.0 * (radius - r) / prob.xi
    return 0.5 + 0.5 * np.tanh(s) if heavy_inside else 0.5 - 0.5 * np.tanh(s)


def cylinder_phi(prob: Problem, centre_xy: Sequence[float], radius: float, heavy_inside: bool) -> np.ndarray:
    """phi0 of a cylinder along z (for quasi-2-D boxes)."""
    z, y, x = np.meshgrid(
        np.arange(prob.nz) + 0.5, np.arange(prob.ny) + 0.5, np.arange(prob.nx) + 0.5, indexing="ij"
    )
    dx = _axis_delta(x, centre_xy[0], prob.nx, not prob.wall[0])
    dy = _axis_delta(y, centre_xy[1], prob.ny, not prob.wall[1])
    r = np.sqrt(dx * dx + dy * dy)
    s = 2.0 * (radius - r) / prob.xi
    return 0.5 + 0.5 * np.tanh(s) if heavy_inside else 0.5 - 0.5 * np.tanh(s)


def slab_phi(prob: Problem, x1: float, x2: float, axis: int = 0) -> np.ndarray:
    """Heavy slab x1 < x < x2 along ``axis`` (periodic), tanh profiles at both faces."""
    n = prob.shape[2 - axis]
    c = np.arange(n) + 0.5
    faces = np.array([x1, x2, x1 - n, x2 - n, x1 + n, x2 + n])
    dist = np.abs(c[:, None] - faces[None, :]).min(axis=1)
    signed = np.where((c > x1) & (c < x2), dist, -dist)  # positive inside the heavy slab
    prof = 0.5 + 0.5 * np.tanh(2.0 * signed / prob.xi)
    shape = [1, 1, 1]
    shape[2 - axis] = n
    return np.broadcast_to(prof.reshape(shape), prob.shape).copy()


def many_bubbles_phi(prob: Problem, bubbles: np.ndarray, window: float = 24.0) -> np.ndarray:
    """phi0 = min over bubbles (light inside) of the tanh profile.

    ``bubbles`` is an (n, 4) array of (cx, cy, cz, radius).  Each bubble only
    touches a cube of half-width radius + window cells (beyond it the profile
    rounds to 1 in float32); periodic axes wrap the cube.
    """
    phi = np.ones(prob.shape, dtype=np.float64)
    n = (prob.nx, prob.ny, prob.nz)
    for cx, cy, cz, r in bubbles:
        c = (cx, cy, cz)
        idx, dist = [], []
        for a in range(3):
            lo = int(math.floor(c[a] - r - window))
            hi = int(math.ceil(c[a] + r + window))
            ids = np.arange(lo, hi + 1)
            if prob.wall[a]:
                ids = ids[(ids >= 0) & (ids < n[a])]
                d = ids + 0.5 - c[a]
            else:
                d = ids + 0.5 - c[a]
                ids = np.mod(ids, n[a])
                if hi - lo + 1 > n[a]:  # window wider than the box: keep each cell once
                    ids, first = np.unique(ids, return_index=True)
                    d = _axis_delta(ids + 0.5, c[a], n[a], True)
            idx.append(ids)
            dist.append(d)
        r2 = dist[2][:, None, None] ** 2 + dist[1][None, :, None] ** 2 + dist[0][None, None, :] ** 2
        local = 0.5 - 0.5 * np.tanh(2.0 * (r - np.sqrt(r2)) / prob.xi)
        sub = np.ix_(idx[2], idx[1], idx[0])
        phi[sub] = np.minimum(phi[sub], local)
    return phi


def place_bubbles(prob: Problem, count: int, dmin: float, dmax: float, seed: int = SEED,
                  max_tries: int = 200000) -> np.ndarray:
    """Rejection sampling of non-overlapping bubbles (minimum image on periodic
    axes): centre distance >= r1 + r2 + xi.  Returns (count, 4) = (cx, cy, cz, r)."""
    rng = np.random.default_rng(seed)
    n = np.array([prob.nx, prob.ny, prob.nz], dtype=np.float64)
    periodic = np.array([not w for w in prob.wall])
    out = np.zeros((0, 4))
    tries = 0
    while out.shape[0] < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place all bubbles")
        r = 0.5 * rng.uniform(dmin, dmax)
        lo = np.where(periodic, 0.0, r + 1.0)
        hi = np.where(periodic, n, n - r - 1.0)
        c = rng.uniform(lo, hi)
        if out.shape[0]:
            d = out[:, :3] - c
            d = np.where(periodic, d - n * np.round(d / n), d)
            dist = np.sqrt((d * d).sum(axis=1))
            if np.any(dist < out[:, 3] + r + prob.xi):
                continue
        out = np.vstack([out, np.concatenate([c, [r]])[None, :]])
    return out


# ---------------------------------------------------------------------------
# the named workloads


def _bubble_params(D: float, Eo: float, Mo: float, t_ref: float, rho_H: float = 1.0):
    """gravity, sigma and nu_H from Eo, Mo and t_ref = sqrt(D/g) (Section 6.1 groups)."""
    g = D / (t_ref * t_ref)
    sigma = g * rho_H * D * D / Eo
    re_gr = (Eo ** 3 / Mo) ** 0.25
    mu_H = rho_H * math.sqrt(g * D ** 3) / re_gr
    return g, sigma, mu_H / rho_H


def static_droplet(n: int = 32, radius: float = 8.0, q_hydro: int = 19):
    prob = Problem(n, n, n, wall=(0, 0, 0), q_hydro=q_hydro, rho_H=1.0, rho_ratio=1000.0, nu_H=0.01,
                   mu_ratio=100.0, sigma=1e-4, xi=5.0, mobility=0.02, gravity=(0.0, 0.0, 0.0), rho_ref=1.0)
    phi0 = sphere_phi(prob, (n / 2, n / 2, n / 2), radius, heavy_inside=True)
    return prob, phi0.astype(np.float32)


def rising_bubble(nx: int = 128, ny: int = 512, nz: int = 128, D: float = 32.0, centre=None,
                  Eo: float = 10.0, Mo: float = 1e-3, t_ref: float = 2000.0, q_hydro: int = 27):
    g, sigma, nu_H = _bubble_params(D, Eo, Mo, t_ref)
    prob = Problem(nx, ny, nz, wall=(1, 1, 1), q_hydro=q_hydro, rho_H=1.0, rho_ratio=1000.0, nu_H=nu_H,
                   mu_ratio=100.0, sigma=sigma, xi=5.0, mobility=0.04, gravity=(0.0, -g, 0.0), rho_ref=1.0,
                   clamp_phi=1, store_phi_ref=1.0)
    if centre is None:
        centre = (nx / 2, 2 * D, nz / 2)
    phi0 = sphere_phi(prob, centre, D / 2, heavy_inside=False)
    return prob, phi0.astype(np.float32)


def precision_bubble():
    return rising_bubble(64, 64, 64, D=16.0, centre=(32.0, 16.0, 32.0), t_ref=1000.0)


def precision_timing(n: int = 512):
    """The box the storage formats are timed on: the rising-bubble parameters
    (D = 32, Eo 10, Mo 1e-3, t_ref 2000, density ratio 1000) on an n^3 box walled
    on every face, the bubble at (n/2, 64, n/2)."""
    return rising_bubble(n, n, n, D=32.0, centre=(n / 2, 64.0, n / 2), t_ref=2000.0)


BATCH_SIZES = ((32, 32, 32), (48, 96, 48), (64, 128, 64), (96, 192, 96))


def _s_nu(nu: float) -> float:
    return 1.0 / (3.0 * nu + 0.5)


def batched(count: int = 64, seed: int = SEED, u_s: float = 0.016, re_gr: float = 30.0):
    """Independent walled rising-bubble problems for batched stepping.

    Each draw: a box among BATCH_SIZES, density ratio among {10, 100, 1000},
    Eo ~ U[1, 50]; bubble diameter D = nx / 4 centred in x and z at height y = 2D.
    With u_s = sqrt(g D) and Re_Gr = rho_H u_s D / mu_H fixed: g = u_s^2 / D,
    sigma = rho_H g D^2 / Eo, nu_H = u_s D / Re_Gr, viscosity ratio 100.  Draws
    whose relaxation rate s_nu = 1 / (3 nu + 1/2) leaves (0.05, 1.98) in either
    fluid are redrawn.  Returns [(Problem, phi0, draw)] with draw = dict(size,
    rho_ratio, Eo, D)."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        size = BATCH_SIZES[int(rng.integers(len(BATCH_SIZES)))]
        ratio = float((10.0, 100.0, 1000.0)[int(rng.integers(3))])
        Eo = float(rng.uniform(1.0, 50.0))
        nx, ny, nz = size
        D = nx / 4.0
        g = u_s * u_s / D
        nu_H = u_s * D / re_gr
        nu_L = nu_H * ratio / 100.0  # mu_L = mu_H / 100, rho_L = rho_H / ratio
        if not all(0.05 < _s_nu(nu) < 1.98 for nu in (nu_H, nu_L)):
            continue
        prob = Problem(nx, ny, nz, wall=(1, 1, 1), q_hydro=27, rho_H=1.0, rho_ratio=ratio, nu_H=nu_H,
                       mu_ratio=100.0, sigma=g * D * D / Eo, xi=5.0, mobility=0.04, gravity=(0.0, -g, 0.0),
                       rho_ref=1.0, clamp_phi=1, store_phi_ref=1.0)
        phi0 = sphere_phi(prob, (nx / 2, 2 * D, nz / 2), D / 2, heavy_inside=False).astype(np.float32)
        out.append((prob, phi0, dict(size=size, rho_ratio=ratio, Eo=Eo, D=D)))
    return out


def roofline2d(nx: int = 8192, ny: int = 16384, radius: float = 12.0, spacing: int = 64):
    """The two-dimensional pair's benchmark box (nx x ny x 1, D2Q9 for both
    lattices, triply periodic): light circles of radius 12 on a square lattice of
    pitch 64 in heavy fluid, the roofline workload's physics (density ratio 1000,
    viscosity ratio 100, sigma 1e-4, xi 5, M 0.02, gravity from Eo 10 at D 24,
    rho_ref the mean density).  134.2 M cells at the default size, as 512^3."""
    sigma, Eo, D_ref = 1e-4, 10.0, 24.0
    g = Eo * sigma / (D_ref * D_ref)
    prob = Problem(nx, ny, 1, wall=(0, 0, 0), q_hydro=9, q_phase=9, rho_H=1.0, rho_ratio=1000.0, nu_H=0.01,
                   mu_ratio=100.0, sigma=sigma, xi=5.0, mobility=0.02, gravity=(0.0, -g, 0.0), clamp_phi=1)
    x = (np.arange(nx) + 0.5) % spacing - spacing / 2
    y = (np.arange(ny) + 0.5) % spacing - spacing / 2
    r = np.sqrt(y[:, None] ** 2 + x[None, :] ** 2).astype(np.float32)
    phi0 = (0.5 - 0.5 * np.tanh(2.0 * (radius - r) / prob.xi)).astype(np.float32)[None]
    mean_phi = float(phi0.astype(np.float64).mean())
    prob.rho_ref = prob.rho_L + mean_phi * (prob.rho_H - prob.rho_L)
    return prob, phi0


def roofline(n: int = 512, count: int = 400, dmin: float = 16.0, dmax: float = 32.0, seed: int = SEED):
    sigma, Eo, D_ref = 1e-4, 10.0, 24.0
    g = Eo * sigma / (1.0 * D_ref * D_ref)
    prob = Problem(n, n, n, wall=(0, 0, 0), q_hydro=27, rho_H=1.0, rho_ratio=1000.0, nu_H=0.01,
                   mu_ratio=100.0, sigma=sigma, xi=5.0, mobility=0.02, gravity=(0.0, -g, 0.0), clamp_phi=1,
                   store_phi_ref=1.0)
    bubbles = place_bubbles(prob, count, dmin, dmax, seed)
    phi0 = many_bubbles_phi(prob, bubbles).astype(np.float32)
    # buoyancy reference: the mean density, so a periodic gravity axis carries no net force
    mean_phi = float(phi0.astype(np.float64).mean())
    prob.rho_ref = prob.rho_L + mean_phi * (prob.rho_H - prob.rho_L)
    return prob, phi0, bubbles


# ---------------------------------------------------------------------------
# random states for one-step parity checks


def random_smooth_field(shape, rng, modes: int = 3, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """A smooth random field in [lo, hi] (sum of a few periodic Fourier modes)."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    f = np.zeros(shape)
    for _ in range(modes):
        k = rng.integers(-2, 3, size=3)
        ph = rng.uniform(0, 2 * np.pi)
        f += rng.normal() * np.cos(2 * np.pi * (k[0] * x / nx + k[1] * y / ny + k[2] * z / nz) + ph)
    f = (f - f.min()) / max(f.max() - f.min(), 1e-12)
    return lo + (hi - lo) * f


def random_state(prob: Problem, seed: int, pop_noise: float = 1e-3):
    """A seeded state (h, g, Phi) of the library's exported layout: h (q_phase, nz, ny, nx),
    g (q_hydro, nz, ny, nx), Phi (nz, ny, nx), all float32.  Phi is a smooth field in
    [0, 1]; h and g are small random populations around a uniform rest state."""
    rng = np.random.default_rng(seed)
    phi = random_smooth_field(prob.shape, rng).astype(np.float32)
    qp = getattr(prob, "q_phase", 15)
    h = (rng.uniform(0.0, 1.0, size=(qp,) + prob.shape) * (1.0 / qp)).astype(np.float32)
    g = (rng.normal(0.0, pop_noise, size=(prob.q_hydro,) + prob.shape)).astype(np.float32)
    return h, g, phi
