"""FP64 CPU oracle of the conservative Allen-Cahn multiphase LBM (test infrastructure).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``acm_oracle.c`` (plain C,
compiled with gcc, FP64, no fast-math, no FMA contraction) through ctypes and
shares no code with the CUDA library.

Array conventions (numpy, C order): scalar fields have shape (nz, ny, nx);
population sets (q, nz, ny, nx); vector fields (3, nz, ny, nx).  Direction i
follows the numbering documented in ``acm_oracle.c`` and in the library's
public header (rest, faces, edges, corners; each direction followed by its
opposite).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "acm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libacm_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile acm_oracle.c into a shared library (OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    return compile_source(_SRC, _LIB)


def compile_source(src: str, out: str) -> str:
    """gcc -O2, FP64 as written: no fast-math and no FMA contraction."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC", src,
            "-o", out + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(out + ".tmp", out)
    return out


class orc_problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("wall", ctypes.c_int * 3),
        ("q_hydro", ctypes.c_int),
        ("rho_H", ctypes.c_double), ("rho_L", ctypes.c_double),
        ("nu_H", ctypes.c_double), ("nu_L", ctypes.c_double),
        ("sigma", ctypes.c_double), ("xi", ctypes.c_double), ("mobility", ctypes.c_double),
        ("gravity", ctypes.c_double * 3),
        ("rho_ref", ctypes.c_double),
        ("theta_from_local_phi", ctypes.c_int),
        ("clamp_phi", ctypes.c_int),
        ("phase_mrt", ctypes.c_int),
        ("q_phase", ctypes.c_int),
    ]


def _bind(cdll):
    P = ctypes.POINTER(orc_problem)
    D = ctypes.POINTER(ctypes.c_double)
    cdll.orc_lattice_table.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), D,
                                       ctypes.POINTER(ctypes.c_int)]
    cdll.orc_derived.argtypes = [P, D]
    cdll.orc_gradient_laplacian.argtypes = [P, ctypes.c_int, D, D, D]
    cdll.orc_phase_cell.argtypes = [P, D, D, D, D, D]
    cdll.orc_hydro_cell.argtypes = [P, D, D, D, D, D]
    cdll.orc_phase_step.argtypes = [P, D, D, D, D, D]
    cdll.orc_hydro_step.argtypes = [P, D, D, D, D]
    cdll.orc_fields.argtypes = [P, D, D, D, D]
    cdll.orc_init.argtypes = [P, D, D, D, D, D]
    cdll.orc_run.argtypes = [P, D, D, D, D, ctypes.c_long]
    cdll.orc_run.restype = ctypes.c_int
    cdll.orc_set_threads.argtypes = [ctypes.c_int]
    cdll.orc_get_threads.restype = ctypes.c_int
    return cdll


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
        return _lib


class using_library:
    """Context manager: route every call of this module to another compiled copy
    of the oracle (the mutation tests build copies with planted mistakes)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        lib()
        self.saved = _lib
        _lib = _bind(ctypes.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_problem(prob, theta_from_local_phi: bool = False, clamp_phi=None, phase_mrt=None) -> orc_problem:
    """Builds the C problem record from a ``workloads.Problem``-like object."""
    p = orc_problem()
    p.nx, p.ny, p.nz = int(prob.nx), int(prob.ny), int(prob.nz)
    for a in range(3):
        p.wall[a] = int(prob.wall[a])
        p.gravity[a] = float(prob.gravity[a])
    p.q_hydro = int(prob.q_hydro)
    p.rho_H, p.rho_L = float(prob.rho_H), float(prob.rho_L)
    p.nu_H, p.nu_L = float(prob.nu_H), float(prob.nu_L)
    p.sigma, p.xi, p.mobility = float(prob.sigma), float(prob.xi), float(prob.mobility)
    p.rho_ref = float(prob.rho_ref)
    p.theta_from_local_phi = int(theta_from_local_phi)
    p.clamp_phi = int(getattr(prob, "clamp_phi", 0) if clamp_phi is None else clamp_phi)
    p.phase_mrt = int(getattr(prob, "phase_mrt", 0) if phase_mrt is None else phase_mrt)
    p.q_phase = int(getattr(prob, "q_phase", 15))
    return p


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def lattice(q: int):
    """(e (q,3) int, w (q,) float64, opp (q,) int) of D2Q9, D3Q15, D3Q19 or D3Q27."""
    e = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q, dtype=np.float64)
    opp = np.zeros(q, dtype=np.int32)
    r = lib().orc_lattice_table(q, e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w),
                                opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if r != q:
        raise ValueError(f"unknown lattice D3Q{q}")
    return e, w, opp


def derived(p: orc_problem) -> dict:
    out = np.zeros(5)
    lib().orc_derived(ctypes.byref(p), _dp(out))
    return dict(tau_H=out[0], tau_L=out[1], omega_phi=out[2], beta=out[3], kappa=out[4])


def gradient_laplacian(p: orc_problem, q: int, phi: np.ndarray):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    grad = np.zeros((3,) + phi.shape)
    lap = np.zeros(phi.shape)
    if lib().orc_gradient_laplacian(ctypes.byref(p), q, _dp(phi), _dp(grad), _dp(lap)) != 0:
        raise ValueError(q)
    return grad, lap


def phase_cell(p: orc_problem, h: np.ndarray, nbprev: np.ndarray, u: np.ndarray):
    h = np.ascontiguousarray(h, dtype=np.float64)
    nb = np.ascontiguousarray(nbprev, dtype=np.float64).reshape(27)
    u = np.ascontiguousarray(u, dtype=np.float64)
    hs = np.zeros(p.q_phase or 15)
    phi = np.zeros(1)
    lib().orc_phase_cell(ctypes.byref(p), _dp(h), _dp(nb), _dp(u), _dp(hs), _dp(phi))
    return hs, float(phi[0])


def hydro_cell(p: orc_problem, g: np.ndarray, nb: np.ndarray):
    """Returns (g*, u, aux) with aux = rho, p*, s_nu, tau, F(3), mu_phi, F_mu(3)."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    nb = np.ascontiguousarray(nb, dtype=np.float64).reshape(27)
    gs = np.zeros(p.q_hydro)
    u = np.zeros(3)
    aux = np.zeros(11)
    lib().orc_hydro_cell(ctypes.byref(p), _dp(g), _dp(nb), _dp(gs), _dp(u), _dp(aux))
    return gs, u, aux


def phase_step(p: orc_problem, h, phi_prev, u_prev):
    h = np.ascontiguousarray(h, dtype=np.float64)
    phi_prev = np.ascontiguousarray(phi_prev, dtype=np.float64)
    u_prev = np.ascontiguousarray(u_prev, dtype=np.float64)
    h_next = np.zeros_like(h)
    phi_now = np.zeros_like(phi_prev)
    lib().orc_phase_step(ctypes.byref(p), _dp(h), _dp(phi_prev), _dp(u_prev), _dp(h_next), _dp(phi_now))
    return h_next, phi_now


def hydro_step(p: orc_problem, g, phi):
    g = np.ascontiguousarray(g, dtype=np.float64)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    g_next = np.zeros_like(g)
    u = np.zeros((3,) + phi.shape)
    lib().orc_hydro_step(ctypes.byref(p), _dp(g), _dp(phi), _dp(g_next), _dp(u))
    return g_next, u


def fields(p: orc_problem, g, phi):
    """(u, p) from (g^k, Phi^k)."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    u = np.zeros((3,) + phi.shape)
    pr = np.zeros(phi.shape)
    lib().orc_fields(ctypes.byref(p), _dp(g), _dp(phi), _dp(u), _dp(pr))
    return u, pr


class State:
    """Oracle state before time step k: h^k, g^k, Phi^{k-1}, u_{k-1}."""

    def __init__(self, p: orc_problem, phi0: np.ndarray):
        self.p = p
        shape = (p.nz, p.ny, p.nx)
        phi0 = np.ascontiguousarray(phi0, dtype=np.float64).reshape(shape)
        self.h = np.zeros((p.q_phase or 15,) + shape)
        self.g = np.zeros((p.q_hydro,) + shape)
        self.phi_prev = np.zeros(shape)
        self.u_prev = np.zeros((3,) + shape)
        lib().orc_init(ctypes.byref(p), _dp(phi0), _dp(self.h), _dp(self.g), _dp(self.phi_prev),
                       _dp(self.u_prev))
        self.k = 0

    def run(self, nsteps: int) -> "State":
        if nsteps > 0:
            r = lib().orc_run(ctypes.byref(self.p), _dp(self.h), _dp(self.g), _dp(self.phi_prev),
                              _dp(self.u_prev), int(nsteps))
            if r != 0:
                raise MemoryError("oracle run failed")
            self.k += nsteps
        return self

    def phi(self) -> np.ndarray:
        """Phi^k = sum_i h_i^k."""
        return self.h.sum(axis=0)

    def fields(self):
        """(phi, u, p) after k steps: phi = sum h^k, u and p from (g^k, Phi^k)."""
        phi = self.phi()
        u, pr = fields(self.p, self.g, phi)
        return phi, u, pr


DIAGNOSTIC_NAMES = ("mass", "mom_x", "mom_y", "mom_z", "light_vol", "light_x", "light_y", "light_z", "light_ux",
                    "light_uy", "light_uz", "max_u")


def diagnostics(prob, phi, u) -> dict:
    """Diagnostics of a state from its fields (FP64 sums, plain numpy).

    The quantities Section 6.1 follows for a rising bubble -- the light phase's
    centroid and its velocity -- plus the conserved phase mass and the momentum:

    * mass          sum phi (conserved by the phase step, Section 3.1);
    * mom_a         sum rho u_a, rho = rho_L + phi (rho_H - rho_L) (eq:density),
                    phi clamped to [0, 1] there when the problem clamps it;
    * light_vol     sum b with the bubble indicator b = clamp(1 - 2 phi, 0, 1):
                    1 in the light phase, 0 from the interface's mid-level
                    phi = 1/2 on, so the heavy bulk does not enter;
    * light_a       sum (a + 1/2) b / sum b, cell centres at i + 1/2 (centroid);
    * light_ua      sum u_a b / sum b (the bubble's mean velocity);
    * max_u         max |u|.

    ``phi`` has shape (nz, ny, nx) and ``u`` (3, nz, ny, nx)."""
    phi = np.asarray(phi, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    nz, ny, nx = phi.shape
    rho_L = float(prob.rho_L)
    f = np.clip(phi, 0.0, 1.0) if getattr(prob, "clamp_phi", 0) else phi
    rho = rho_L + f * (float(prob.rho_H) - rho_L)
    b = np.clip(1.0 - 2.0 * phi, 0.0, 1.0)
    vol = b.sum()
    centre = (np.arange(nx) + 0.5, np.arange(ny) + 0.5, np.arange(nz) + 0.5)
    out = {"mass": phi.sum()}
    for a, name in enumerate("xyz"):
        out["mom_" + name] = (rho * u[a]).sum()
    out["light_vol"] = vol
    # sum over the other two axes first: sum_c (a_c + 1/2) b_c
    per_axis = (b.sum(axis=(0, 1)), b.sum(axis=(0, 2)), b.sum(axis=(1, 2)))
    for a, name in enumerate("xyz"):
        out["light_" + name] = float((centre[a] * per_axis[a]).sum() / vol) if vol > 0 else 0.0
    for a, name in enumerate("xyz"):
        out["light_u" + name] = float((u[a] * b).sum() / vol) if vol > 0 else 0.0
    out["max_u"] = float(np.sqrt((u * u).sum(axis=0)).max())
    return {k: float(out[k]) for k in DIAGNOSTIC_NAMES}
