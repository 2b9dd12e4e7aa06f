"""Rising-bubble observables (Section 6.1): the light phase's centroid and rise
velocity over time, its terminal velocity, and the drag coefficient against the
empirical correlation the paper compares with (eq:analytical_drag_coeff).

The per-step quantities come from the library's FP64 reductions (lbm_reduce:
centroid and velocity weighted by the bubble indicator clamp(1 - 2 phi, 0, 1));
what is here is host arithmetic on a handful of doubles.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def gravity_reynolds(rho_H: float, g: float, D: float, mu_H: float) -> float:
    """Re_Gr = rho_H sqrt(g D^3) / mu_H (Section 6.1)."""
    return rho_H * math.sqrt(g * D ** 3) / mu_H


def eotvos(rho_H: float, g: float, D: float, sigma: float) -> float:
    """Eo = g rho_H D^2 / sigma (Section 6.1)."""
    return g * rho_H * D * D / sigma


def reference_time(D: float, g: float) -> float:
    """t_ref = sqrt(D / g); t* = t / t_ref (Section 6.1)."""
    return math.sqrt(D / g)


def drag_coefficient(g: float, rho_H: float, rho_L: float, D: float, u_t: float) -> float:
    """C_D from the terminal velocity: 4/3 g (rho_H - rho_L) D / (rho_H u_t^2)
    (Section 6.1): buoyancy of a sphere of diameter D balanced by a drag
    C_D rho_H u_t^2 / 2 over its cross-section."""
    return 4.0 / 3.0 * g * (rho_H - rho_L) * D / (rho_H * u_t * u_t)


def drag_correlation(Re: float) -> float:
    """Bhaga and Weber's empirical drag coefficient (eq:analytical_drag_coeff):
    [2.67^(9/10) + (16/Re)^(9/10)]^(10/9) -- Stokes-like 16/Re at small Re, the
    constant 2.67 of spherical-cap bubbles at large Re."""
    return (2.67 ** 0.9 + (16.0 / Re) ** 0.9) ** (10.0 / 9.0)


@dataclass
class RiseRecord:
    """Time series of the light phase: step, centroid (x, y, z) and mean velocity
    (x, y, z), both weighted by the bubble indicator, its volume, max |u|."""
    t: list = field(default_factory=list)
    centroid: list = field(default_factory=list)
    velocity: list = field(default_factory=list)
    volume: list = field(default_factory=list)
    max_u: list = field(default_factory=list)

    def add(self, t: int, d: dict):
        self.t.append(int(t))
        self.centroid.append((d["light_x"], d["light_y"], d["light_z"]))
        self.velocity.append((d["light_ux"], d["light_uy"], d["light_uz"]))
        self.volume.append(d["light_vol"])
        self.max_u.append(d["max_u"])

    def arrays(self):
        return (np.asarray(self.t, dtype=np.float64), np.asarray(self.centroid), np.asarray(self.velocity),
                np.asarray(self.volume), np.asarray(self.max_u))


def track(sim, steps: int, every: int = 100, record: RiseRecord | None = None) -> RiseRecord:
    """Steps `sim` (anything with step(n), reduce() and steps_done()) `steps`
    times, recording the light phase every `every` steps (and at the start)."""
    rec = record if record is not None else RiseRecord()
    if not rec.t:
        rec.add(sim.steps_done(), sim.reduce())
    done = 0
    while done < steps:
        n = min(every, steps - done)
        sim.step(n)
        done += n
        rec.add(sim.steps_done(), sim.reduce())
    return rec


def terminal_velocity(rec: RiseRecord, t_ref: float, window: float = 2.0, axis: int = 1):
    """Rise velocity over the last `window` reference times: the slope of a
    least-squares line through the centroid's height (the bubble's translation
    velocity), and its steadiness, |slope(second half) - slope(first half)| /
    slope."""
    t, c, _, _, _ = rec.arrays()
    sel = t >= t[-1] - window * t_ref
    ts, ys = t[sel], c[sel, axis]
    if len(ts) < 4:
        raise ValueError("terminal_velocity needs at least 4 records in the window")
    slope = float(np.polyfit(ts, ys, 1)[0])
    h = len(ts) // 2
    s1, s2 = np.polyfit(ts[:h + 1], ys[:h + 1], 1)[0], np.polyfit(ts[h:], ys[h:], 1)[0]
    return slope, float(abs(s2 - s1) / abs(slope)) if slope != 0.0 else math.inf


def mean_core_velocity(rec: RiseRecord, t_ref: float, window: float = 2.0, axis: int = 1) -> float:
    """The indicator-weighted mean velocity averaged over the window.  It weights
    the bubble's core, whose internal circulation moves faster than the bubble,
    so it exceeds the translation velocity (a diagnostic, not u_t)."""
    t, _, vel, _, _ = rec.arrays()
    return float(vel[t >= t[-1] - window * t_ref, axis].mean())


def centroid_velocity(rec: RiseRecord, axis: int = 1) -> np.ndarray:
    """d(centroid)/dt by central differences of the recorded centroid (a check on
    the directly averaged velocity)."""
    t, c, _, _, _ = rec.arrays()
    return np.gradient(c[:, axis], t)


def summary(prob, rec: RiseRecord, D: float, window: float = 2.0) -> dict:
    """Dimensionless groups, terminal velocity, terminal Reynolds number and drag
    coefficient of a rising-bubble run of `prob` (a workloads.Problem with gravity
    along -y) recorded in `rec`."""
    g = -prob.gravity[1]
    mu_H = prob.rho_H * prob.nu_H
    t_ref = reference_time(D, g)
    u_t, spread = terminal_velocity(rec, t_ref, window)
    re_gr = gravity_reynolds(prob.rho_H, g, D, mu_H)
    re_t = prob.rho_H * u_t * D / mu_H
    t, c, _, vol, _ = rec.arrays()
    return {
        "D": D, "Eo": eotvos(prob.rho_H, g, D, prob.sigma), "Re_Gr": re_gr, "t_ref": t_ref,
        "t_star_end": float(t[-1] / t_ref), "u_t": u_t, "u_t_steadiness": spread, "Re_t": re_t,
        "u_core_mean": mean_core_velocity(rec, t_ref, window),
        "C_D": drag_coefficient(g, prob.rho_H, prob.rho_L, D, u_t),
        "C_D_correlation_Re_Gr": drag_correlation(re_gr), "C_D_correlation_Re_t": drag_correlation(re_t),
        "centroid_rise": float(c[-1, 1] - c[0, 1]), "light_volume_drift": float(vol[-1] / vol[0] - 1.0),
    }
