"""ctypes binding of the C ABI in include/lbm.h (argument marshalling only).

The functions below carry the C names and forward plain pointers and sizes;
every computation runs in the CUDA library.  ``Simulation`` is a small
convenience wrapper that takes its device workspace and its stream from
PyTorch.  There is no CPU fallback: if the library is not built, loading
raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

from . import _build

LBM_OK, LBM_ERR_ARG, LBM_ERR_CUDA, LBM_ERR_OOM, LBM_ERR_DIVERGED, LBM_ERR_STATE = 0, -1, -2, -3, -4, -5
STATUS_NAMES = {0: "LBM_OK", -1: "LBM_ERR_ARG", -2: "LBM_ERR_CUDA", -3: "LBM_ERR_OOM", -4: "LBM_ERR_DIVERGED",
                -5: "LBM_ERR_STATE"}
LBM_PRECISION_FP32, LBM_PRECISION_FP16, LBM_PRECISION_BF16 = 0, 1, 2
LBM_PHASE_SRT, LBM_PHASE_MRT = 0, 1
LBM_FORM_FUSED, LBM_FORM_UNFUSED, LBM_FORM_FUSED_CELL, LBM_FORM_FUSED_PAIR = 0, 1, 2, 3
FORMS = {"fused": LBM_FORM_FUSED, "unfused": LBM_FORM_UNFUSED, "cell": LBM_FORM_FUSED_CELL, "pair": LBM_FORM_FUSED_PAIR}
PRECISIONS = {"fp32": LBM_PRECISION_FP32, "fp16": LBM_PRECISION_FP16, "bf16": LBM_PRECISION_BF16}
DIAG_NAMES = ["mass", "mom_x", "mom_y", "mom_z", "light_vol", "light_x", "light_y", "light_z", "light_ux",
              "light_uy", "light_uz", "max_u"]
LBM_DIAG_COUNT = len(DIAG_NAMES)


class lbm_domain(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("wall", ctypes.c_int * 3),
                ("q_phase", ctypes.c_int), ("q_hydro", ctypes.c_int)]


class lbm_params(ctypes.Structure):
    _fields_ = [("rho_H", ctypes.c_double), ("rho_ratio", ctypes.c_double), ("nu_H", ctypes.c_double),
                ("mu_ratio", ctypes.c_double), ("sigma", ctypes.c_double), ("xi", ctypes.c_double),
                ("mobility", ctypes.c_double), ("gravity", ctypes.c_double * 3), ("rho_ref", ctypes.c_double),
                ("precision", ctypes.c_int), ("clamp_phi", ctypes.c_int), ("store_phi_ref", ctypes.c_double),
                ("store_g_scale", ctypes.c_double), ("phase_collision", ctypes.c_int),
                ("kernel_form", ctypes.c_int)]


class LBMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None
_lock = threading.Lock()

_VP, _FP, _DP = ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
_SIGNATURES = {
    "lbm_workspace_size": ([ctypes.POINTER(lbm_domain), ctypes.POINTER(lbm_params), ctypes.POINTER(ctypes.c_size_t)],
                           ctypes.c_int),
    "lbm_create": ([ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(lbm_domain), ctypes.POINTER(lbm_params), _VP, _VP,
                    ctypes.c_size_t], ctypes.c_int),
    "lbm_init_phase": ([_VP, _FP, ctypes.c_int], ctypes.c_int),
    "lbm_step": ([_VP, ctypes.c_int64], ctypes.c_int),
    "lbm_get_fields": ([_VP, _FP, _FP, _FP, ctypes.c_int], ctypes.c_int),
    "lbm_reduce": ([_VP, _DP], ctypes.c_int),
    "lbm_get_state": ([_VP, _FP, _FP, _FP, ctypes.c_int], ctypes.c_int),
    "lbm_set_state": ([_VP, _FP, _FP, _FP, ctypes.c_int], ctypes.c_int),
    "lbm_synchronize": ([_VP], ctypes.c_int),
    "lbm_steps_done": ([_VP], ctypes.c_int64),
    "lbm_last_error": ([_VP], ctypes.c_char_p),
    "lbm_destroy": ([_VP], None),
    "lbm_reduce_state_noalloc": ([ctypes.POINTER(lbm_domain), ctypes.POINTER(lbm_params), _FP, _FP, _DP, _VP],
                                 ctypes.c_int),
    "lbm_batch_workspace_size": ([ctypes.c_int, ctypes.POINTER(lbm_domain), ctypes.POINTER(lbm_params),
                                  ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "lbm_batch_create": ([ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(lbm_domain),
                          ctypes.POINTER(lbm_params), _VP, _VP, ctypes.c_size_t], ctypes.c_int),
    "lbm_batch_size": ([_VP], ctypes.c_int),
    "lbm_batch_member": ([_VP, ctypes.c_int], _VP),
    "lbm_batch_step": ([_VP, ctypes.c_int64], ctypes.c_int),
    "lbm_batch_tune": ([_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _DP], ctypes.c_int),
    "lbm_batch_set_config": ([_VP, ctypes.c_int], ctypes.c_int),
    "lbm_batch_synchronize": ([_VP], ctypes.c_int),
    "lbm_batch_last_error": ([_VP], ctypes.c_char_p),
    "lbm_batch_destroy": ([_VP], None),
}
BATCH_SHAPES = [(4, 2), (8, 1), (2, 4), "pair"]  # the autotuner's tile shapes, in its order: (TY, TZ) of
# 32 x TY x TZ cells with one cell per thread, and "pair", 32 x 4 x 2 cells with two cells per thread
BATCH_ORDERS = ["member", "round_robin"]
BATCH_HALOS = ["loads", "tma"]  # phi halo staging: per-thread loads, or one TMA tensor copy per block


def batch_choice(shape, order, halo="loads") -> int:
    """Candidate index of lbm_batch_tune / lbm_batch_set_config."""
    shape = shape if isinstance(shape, str) else tuple(shape)
    return (BATCH_HALOS.index(halo) * len(BATCH_SHAPES) + BATCH_SHAPES.index(shape)) * len(BATCH_ORDERS) + \
        BATCH_ORDERS.index(order)


def batch_tile_name(shape) -> str:
    """Cells of a tile shape, e.g. "32x4x2", and "32x4x2/pair" for the two-cell tile."""
    return "32x4x2/pair" if shape == "pair" else f"32x{shape[0]}x{shape[1]}"


def batch_candidate(choice: int):
    """(shape (TY, TZ), order name, halo name) of a candidate index."""
    no, ns = len(BATCH_ORDERS), len(BATCH_SHAPES)
    return BATCH_SHAPES[(choice // no) % ns], BATCH_ORDERS[choice % no], BATCH_HALOS[choice // (no * ns)]


def header_functions() -> list:
    """Names of the functions declared in include/lbm.h."""
    text = open(os.path.join(_build.INCLUDE, "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", text)))


def library_path() -> str:
    return _build.LIBRARY


def load():
    """Loads liblbm.so (built by ``__graft_entry__.build()``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIBRARY):
                raise RuntimeError(f"CUDA library not built: {_build.LIBRARY} (run __graft_entry__.build())")
            lib = ctypes.CDLL(_build.LIBRARY)
            for name, (args, res) in _SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
        return _lib


def _check(status: int, handle=None):
    if status != LBM_OK:
        msg = load().lbm_last_error(handle)
        raise LBMError(status, msg.decode() if msg else "")


def _check_batch(status: int, b):
    if status != LBM_OK:
        msg = load().lbm_batch_last_error(b)
        raise LBMError(status, msg.decode() if msg else "")


def make_domain(nx, ny, nz, wall=(0, 0, 0), q_hydro=27, q_phase=15) -> lbm_domain:
    d = lbm_domain()
    d.nx, d.ny, d.nz = int(nx), int(ny), int(nz)
    for a in range(3):
        d.wall[a] = int(wall[a])
    d.q_phase, d.q_hydro = int(q_phase), int(q_hydro)
    return d


def make_params(rho_H=1.0, rho_ratio=1000.0, nu_H=0.01, mu_ratio=100.0, sigma=1e-4, xi=5.0, mobility=0.02,
                gravity=(0.0, 0.0, 0.0), rho_ref=0.0, precision=LBM_PRECISION_FP32, clamp_phi=0, store_phi_ref=0.0,
                store_g_scale=0.0, phase_collision=LBM_PHASE_SRT, kernel_form=LBM_FORM_FUSED) -> lbm_params:
    p = lbm_params()
    p.rho_H, p.rho_ratio, p.nu_H, p.mu_ratio = float(rho_H), float(rho_ratio), float(nu_H), float(mu_ratio)
    p.sigma, p.xi, p.mobility = float(sigma), float(xi), float(mobility)
    for a in range(3):
        p.gravity[a] = float(gravity[a])
    p.rho_ref, p.precision, p.clamp_phi = float(rho_ref), int(precision), int(clamp_phi)
    p.store_phi_ref, p.store_g_scale = float(store_phi_ref), float(store_g_scale)
    p.phase_collision = int(phase_collision)
    p.kernel_form = int(kernel_form)
    return p


def from_problem(prob, precision=None, form=None):
    """(lbm_domain, lbm_params) of a ``workloads.Problem``-like object; ``precision``
    ("fp32", "fp16", "bf16" or an LBM_PRECISION_* value) overrides the problem's,
    ``form`` ("fused", "unfused", "cell", "pair" or an LBM_FORM_* value) its kernel
    form."""
    d = make_domain(prob.nx, prob.ny, prob.nz, prob.wall, prob.q_hydro, getattr(prob, "q_phase", 15))
    prec = getattr(prob, "precision", "fp32") if precision is None else precision
    prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    p = make_params(prob.rho_H, prob.rho_ratio, prob.nu_H, prob.mu_ratio, prob.sigma, prob.xi, prob.mobility,
                    prob.gravity, prob.rho_ref, precision=prec, clamp_phi=int(getattr(prob, "clamp_phi", 0)),
                    store_phi_ref=float(getattr(prob, "store_phi_ref", 0.0)),
                    phase_collision=LBM_PHASE_MRT if getattr(prob, "phase_mrt", 0) else LBM_PHASE_SRT,
                    kernel_form=LBM_FORM_UNFUSED if getattr(prob, "unfused", 0) else LBM_FORM_FUSED)
    if form is not None:
        p.kernel_form = FORMS[form] if isinstance(form, str) else int(form)
    return d, p


# ---- the C functions, same names, pointers as Python ints -------------------------------------------


def lbm_workspace_size(dom: lbm_domain, prm: lbm_params) -> int:
    n = ctypes.c_size_t(0)
    _check(load().lbm_workspace_size(ctypes.byref(dom), ctypes.byref(prm), ctypes.byref(n)))
    return n.value


def lbm_create(dom: lbm_domain, prm: lbm_params, stream: int = 0, workspace: int = 0, workspace_bytes: int = 0):
    h = ctypes.c_void_p()
    _check(load().lbm_create(ctypes.byref(h), ctypes.byref(dom), ctypes.byref(prm), stream or None, workspace or None,
                             workspace_bytes))
    return h


def lbm_init_phase(h, phi0: int, on_device: int):
    _check(load().lbm_init_phase(h, phi0, on_device), h)


def lbm_step(h, n: int):
    _check(load().lbm_step(h, int(n)), h)


def lbm_get_fields(h, phi: int, u: int, p: int, on_device: int):
    _check(load().lbm_get_fields(h, phi or None, u or None, p or None, on_device), h)


def lbm_reduce(h) -> np.ndarray:
    out = np.zeros(LBM_DIAG_COUNT)
    _check(load().lbm_reduce(h, out.ctypes.data_as(_DP)), h)
    return out


def lbm_get_state(h, hp: int, gp: int, phip: int, on_device: int):
    _check(load().lbm_get_state(h, hp or None, gp or None, phip or None, on_device), h)


def lbm_set_state(h, hp: int, gp: int, phip: int, on_device: int):
    _check(load().lbm_set_state(h, hp, gp, phip, on_device), h)


def lbm_synchronize(h):
    _check(load().lbm_synchronize(h), h)


def lbm_steps_done(h) -> int:
    return int(load().lbm_steps_done(h))


def lbm_last_error(h=None) -> str:
    m = load().lbm_last_error(h)
    return m.decode() if m else ""


def lbm_destroy(h):
    load().lbm_destroy(h)


def lbm_reduce_state_noalloc(dom: lbm_domain, prm: lbm_params, g: int, phi: int, stream: int = 0) -> np.ndarray:
    """Diagnostics of a device-resident state (g natural layout, phi) without any
    device allocation by the library; see include/lbm.h."""
    out = np.zeros(LBM_DIAG_COUNT)
    _check(load().lbm_reduce_state_noalloc(ctypes.byref(dom), ctypes.byref(prm), g, phi, out.ctypes.data_as(_DP),
                                           stream or None))
    return out


def _arrays(doms, prms):
    n = len(doms)
    if n != len(prms) or n < 1:
        raise ValueError("need as many parameter sets as domains, at least one")
    return n, (lbm_domain * n)(*doms), (lbm_params * n)(*prms)


def lbm_batch_workspace_size(doms, prms) -> int:
    n, da, pa = _arrays(doms, prms)
    out = ctypes.c_size_t(0)
    _check(load().lbm_batch_workspace_size(n, da, pa, ctypes.byref(out)))
    return out.value


def lbm_batch_create(doms, prms, stream: int = 0, workspace: int = 0, workspace_bytes: int = 0):
    n, da, pa = _arrays(doms, prms)
    b = ctypes.c_void_p()
    _check(load().lbm_batch_create(ctypes.byref(b), n, da, pa, stream or None, workspace or None, workspace_bytes))
    return b


def lbm_batch_size(b) -> int:
    return int(load().lbm_batch_size(b))


def lbm_batch_member(b, i: int):
    h = load().lbm_batch_member(b, int(i))
    if not h:
        raise IndexError(f"batch has no member {i}")
    return ctypes.c_void_p(h)


def lbm_batch_step(b, n: int):
    _check_batch(load().lbm_batch_step(b, int(n)), b)


def lbm_batch_tune(b, trial_steps: int = 5):
    """(choice, ms_per_step[6]) -- choice = shape * 2 + order."""
    choice = ctypes.c_int(-1)
    ms = np.zeros(len(BATCH_HALOS) * len(BATCH_SHAPES) * len(BATCH_ORDERS))
    _check_batch(load().lbm_batch_tune(b, int(trial_steps), ctypes.byref(choice), ms.ctypes.data_as(_DP)), b)
    return choice.value, ms


def lbm_batch_set_config(b, choice: int):
    _check_batch(load().lbm_batch_set_config(b, int(choice)), b)


def lbm_batch_synchronize(b):
    _check_batch(load().lbm_batch_synchronize(b), b)


def lbm_batch_last_error(b) -> str:
    m = load().lbm_batch_last_error(b)
    return m.decode() if m else ""


def lbm_batch_destroy(b):
    load().lbm_batch_destroy(b)


# ---- convenience wrapper: device memory and stream from PyTorch --------------------------------------


class Simulation:
    """One simulation on the current CUDA device.  Workspace = a torch uint8
    tensor; all work goes to torch's current stream (or ``stream``)."""

    def __init__(self, domain: lbm_domain, params: lbm_params, stream=None, device=None, _member_of=None):
        import torch

        self.torch = torch
        if _member_of is not None:  # a member of a Batch: the batch owns handle and memory
            batch, i = _member_of
            self.domain, self.params, self.device, self.stream = domain, params, batch.device, batch.stream
            self._batch = batch
            self.handle = lbm_batch_member(batch.handle, i)
            self.shape = (domain.nz, domain.ny, domain.nx)
            self.N = domain.nx * domain.ny * domain.nz
            return
        self._batch = None
        self.domain, self.params = domain, params
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.nbytes = lbm_workspace_size(domain, params)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=self.device)
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            base = self.workspace.data_ptr()
            aligned = (base + 255) & ~255
            self.handle = lbm_create(domain, params, self.stream.cuda_stream, aligned, self.nbytes)
        self.shape = (domain.nz, domain.ny, domain.nx)
        self.N = domain.nx * domain.ny * domain.nz

    @classmethod
    def from_problem(cls, prob, precision=None, form=None, **kw):
        d, p = from_problem(prob, precision, form)
        return cls(d, p, **kw)

    def close(self):
        if getattr(self, "_batch", None) is not None:  # members go with their batch
            self.handle = None
            return
        if getattr(self, "handle", None):
            lbm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, t):
        assert t.is_cuda and t.is_contiguous() and t.dtype == self.torch.float32
        return t.data_ptr()

    def init_phase(self, phi0):
        if isinstance(phi0, np.ndarray):
            a = np.ascontiguousarray(phi0, dtype=np.float32)
            assert a.size == self.N
            lbm_init_phase(self.handle, a.ctypes.data, 0)
        else:
            assert phi0.numel() == self.N
            lbm_init_phase(self.handle, self._dev(phi0), 1)

    def step(self, n: int = 1):
        lbm_step(self.handle, n)

    def steps_done(self) -> int:
        return lbm_steps_done(self.handle)

    def synchronize(self):
        lbm_synchronize(self.handle)

    def fields(self, on_device: bool = True):
        """(phi, u, p) as torch tensors (device) or numpy arrays (host)."""
        if on_device:
            t = self.torch
            phi = t.empty(self.shape, device=self.device)
            u = t.empty((3,) + self.shape, device=self.device)
            p = t.empty(self.shape, device=self.device)
            lbm_get_fields(self.handle, phi.data_ptr(), u.data_ptr(), p.data_ptr(), 1)
            return phi, u, p
        phi = np.empty(self.shape, np.float32)
        u = np.empty((3,) + self.shape, np.float32)
        p = np.empty(self.shape, np.float32)
        lbm_get_fields(self.handle, phi.ctypes.data, u.ctypes.data, p.ctypes.data, 0)
        return phi, u, p

    def reduce(self) -> dict:
        return dict(zip(DIAG_NAMES, lbm_reduce(self.handle)))

    def get_state(self, on_device: bool = False):
        q, qp = self.domain.q_hydro, self.domain.q_phase
        if on_device:
            t = self.torch
            h = t.empty((qp,) + self.shape, device=self.device)
            g = t.empty((q,) + self.shape, device=self.device)
            phi = t.empty(self.shape, device=self.device)
            lbm_get_state(self.handle, h.data_ptr(), g.data_ptr(), phi.data_ptr(), 1)
            return h, g, phi
        h = np.empty((qp,) + self.shape, np.float32)
        g = np.empty((q,) + self.shape, np.float32)
        phi = np.empty(self.shape, np.float32)
        lbm_get_state(self.handle, h.ctypes.data, g.ctypes.data, phi.ctypes.data, 0)
        return h, g, phi

    def set_state(self, h, g, phi):
        if isinstance(h, np.ndarray):
            h = np.ascontiguousarray(h, dtype=np.float32)
            g = np.ascontiguousarray(g, dtype=np.float32)
            phi = np.ascontiguousarray(phi, dtype=np.float32)
            assert h.size == self.domain.q_phase * self.N and g.size == self.domain.q_hydro * self.N
            assert phi.size == self.N
            lbm_set_state(self.handle, h.ctypes.data, g.ctypes.data, phi.ctypes.data, 0)
        else:
            lbm_set_state(self.handle, self._dev(h), self._dev(g), self._dev(phi), 1)


class Batch:
    """Independent simulations stepped together (``lbm_batch_*``).  One torch
    workspace holds every member; ``members[i]`` is a ``Simulation`` view of
    member i for initialisation and read-back (do not step it on its own)."""

    def __init__(self, domains, params, stream=None, device=None):
        import torch

        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.nbytes = lbm_batch_workspace_size(domains, params)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=self.device)
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            aligned = (self.workspace.data_ptr() + 255) & ~255
            self.handle = lbm_batch_create(domains, params, self.stream.cuda_stream, aligned, self.nbytes)
        self.members = [Simulation(d, p, _member_of=(self, i)) for i, (d, p) in enumerate(zip(domains, params))]
        self.cells = sum(d.nx * d.ny * d.nz for d in domains)

    @classmethod
    def from_problems(cls, problems, **kw):
        dp = [from_problem(p) for p in problems]
        return cls([d for d, _ in dp], [p for _, p in dp], **kw)

    def __len__(self):
        return len(self.members)

    def step(self, n: int = 1):
        lbm_batch_step(self.handle, n)

    def tune(self, trial_steps: int = 5):
        """Times every (halo staging, tile shape, table order) on the batch -- the
        trial steps advance every member -- and keeps the fastest.  Returns
        (shape (TY, TZ), order name, halo name, ms_per_step for all candidates,
        -1 where the TMA staging is unavailable)."""
        choice, ms = lbm_batch_tune(self.handle, trial_steps)
        shape, order, halo = batch_candidate(choice)
        return shape, order, halo, ms

    def configure(self, shape=(4, 2), order="member", halo="loads"):
        """Selects one candidate of the tuner without timing."""
        lbm_batch_set_config(self.handle, batch_choice(shape, order, halo))

    def synchronize(self):
        lbm_batch_synchronize(self.handle)

    def steps_done(self) -> int:
        return self.members[0].steps_done()

    def close(self):
        if getattr(self, "handle", None):
            for m in self.members:
                m.handle = None
            lbm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
