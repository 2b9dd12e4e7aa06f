"""Single rising bubbles (Section 6.1) on the GPU: centroid and rise velocity
over time, terminal velocity and drag coefficient against the empirical
correlation of eq:analytical_drag_coeff.

One (Eo, Re_Gr) pair runs as one simulation; several run together as a batch
(lbm_batch_*), one member per pair.  Prints one JSON object per pair.

    python rising_bubble.py                              # 128x512x128, D 32, Eo 10, Re_Gr 31.6, t* = 5
    python rising_bubble.py --eo 30 --re-gr 10 20 40 80  # a drag sweep at Eo 30
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402


def problems(args):
    eos, res = list(args.eo), list(args.re_gr)
    if len(eos) == 1:
        eos = eos * len(res)
    if len(res) == 1:
        res = res * len(eos)
    if len(eos) != len(res):
        raise SystemExit("--eo and --re-gr need one value or the same number of values")
    nx, ny, nz = args.size
    out = []
    for eo, re in zip(eos, res):
        mo = eo ** 3 / re ** 4  # Re_Gr = (Eo^3 / Mo)^(1/4)
        prob, phi0 = W.rising_bubble(nx, ny, nz, D=args.D, Eo=eo, Mo=mo, t_ref=args.t_ref, q_hydro=args.q)
        if args.rho_ratio:
            prob.rho_ratio = args.rho_ratio
        if args.walls == "top-bottom":  # the paper's setup: periodic sides
            prob.wall = (0, 1, 0)
        out.append((prob, phi0))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--size", type=int, nargs=3, default=[128, 512, 128], metavar=("NX", "NY", "NZ"))
    ap.add_argument("--D", type=float, default=32.0, help="bubble diameter (cells); centre (nx/2, 2D, nz/2)")
    ap.add_argument("--eo", type=float, nargs="+", default=[10.0])
    ap.add_argument("--re-gr", type=float, nargs="+", default=[(10.0 ** 3 / 1e-3) ** 0.25], help="default: Mo 1e-3 at Eo 10")
    ap.add_argument("--rho-ratio", type=float, default=None, help="default 1000 (viscosity ratio 100)")
    ap.add_argument("--t-ref", type=float, default=2000.0, help="sqrt(D/g) in steps")
    ap.add_argument("--t-star", type=float, default=5.0, help="run length in reference times")
    ap.add_argument("--every", type=int, default=100, help="record every this many steps")
    ap.add_argument("--window", type=float, default=1.0, help="terminal-velocity window in reference times")
    ap.add_argument("--q", type=int, default=27, choices=[19, 27])
    ap.add_argument("--walls", default="all", choices=["all", "top-bottom"],
                    help="no-slip walls on every face, or only at the bottom and top (periodic sides)")
    ap.add_argument("--series", action="store_true", help="include the recorded time series")
    args = ap.parse_args(argv)

    import torch

    from paper_2012_06144_gb300 import lbm, observables as O

    probs = problems(args)
    steps = int(round(args.t_star * args.t_ref))
    stream = torch.cuda.Stream()
    if len(probs) == 1:
        sims = [lbm.Simulation.from_problem(probs[0][0], stream=stream)]
        stepper = sims[0]
    else:
        stepper = lbm.Batch.from_problems([p for p, _ in probs], stream=stream)
        sims = stepper.members
    for s, (_, phi0) in zip(sims, probs):
        s.init_phase(phi0)
    recs = [O.RiseRecord() for _ in sims]
    for s, r in zip(sims, recs):
        r.add(s.steps_done(), s.reduce())
    done = 0
    while done < steps:
        n = min(args.every, steps - done)
        stepper.step(n)
        done += n
        for s, r in zip(sims, recs):
            r.add(s.steps_done(), s.reduce())
    stepper.synchronize()
    for (prob, _), r in zip(probs, recs):
        out = O.summary(prob, r, args.D, window=args.window)
        out.update(size=list(args.size), rho_ratio=prob.rho_ratio, steps=steps)
        if args.series:
            t, c, v, _, _ = r.arrays()
            out["series"] = {"t": t.tolist(), "y_c": c[:, 1].tolist(), "u_y": v[:, 1].tolist()}
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
