"""Flow past a cylinder at Re = 100 with variable resolution (Sec. 4.4): the
case runner, and the drag and lift coefficients of Eq. 18.

``run(res, t_end)`` steps ``cases.cylinder2d(res=res)`` -- a D = 1 cylinder
of wall particles at (10, 8) in a periodic 30 x 16 box, far field at
dp = D/res, the wake rectangle [8, 24] x [5, 11] at dp/2 with h blended
over 4 coarse spacings, uniform initial flow (1, 0) -- with the
kick-drift-kick integrator of the library in FP32 to ``t_end``.  The paper's
free-stream boundary is named but not given in it; in its place a fringe
region (Nordstrom, Nordin & Henningson 1999) over x in [24, 29.5] forces the
wake back to the free stream before it re-enters the periodic box upstream
(sph_params.fringe_*).  Every ``every`` steps it records the force of the
fluid on the cylinder averaged over those steps (sph_params.body_force; the
change of sph_diag.body_impulse over the change of sph_diag.time) and the
coefficients of Eq. 18, C_D = 2 F_x / (rho0 U^2 D) and C_L = 2 F_y / (rho0 U^2 D); over the
last ``window`` time units it reports the mean drag, and, from the
coefficients smoothed by a running mean over ``smooth_width`` time units
(the acoustic noise of the weakly compressible method lies far above the
shedding frequency), the lift amplitude and the Strouhal number St = f D / U
from the mean period between upward zero crossings of C_L.  Table 2 of the paper reports C_D = 1.48 +- 0.015,
C_L = +-0.405 and St = 0.178 at D/dp = 80 (context, not a target here).

    python -m paper_2411_13992_gb300.cylinder --res 36 --t 200

prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import Simulation, cases

FRINGE = (4.0, (1.0, 0.0, 0.0), (24.0, 29.5, 2.0, 1.0))   # lambda_max, U_inf, (x0, x1, rise, fall)


def coefficients(F, rho0=1.0, U=1.0, D=1.0):
    """Eq. 18: (C_D, C_L) from the force on the body."""
    return 2.0 * F[0] / (rho0 * U * U * D), 2.0 * F[1] / (rho0 * U * U * D)


def smooth(t: np.ndarray, y: np.ndarray, width: float) -> np.ndarray:
    """Running mean of y over a window of the given width in time: the body
    force of a weakly compressible particle method carries acoustic noise at
    frequencies far above the shedding frequency (c = 10 U), which the
    window removes."""
    out = np.empty_like(y)
    lo = 0
    csum = np.concatenate([[0.0], np.cumsum(y)])
    for k in range(len(t)):
        while t[k] - t[lo] > width:
            lo += 1
        out[k] = (csum[k + 1] - csum[lo]) / (k + 1 - lo)
    return out


def strouhal(t: np.ndarray, cl: np.ndarray, D=1.0, U=1.0):
    """St = f D / U from the mean period between upward zero crossings of
    C_L - mean(C_L) (linear interpolation between samples; pass a smoothed
    signal); None with fewer than two crossings."""
    y = cl - cl.mean()
    k = np.flatnonzero((y[:-1] < 0.0) & (y[1:] >= 0.0))
    if len(k) < 2:
        return None
    tc = t[k] - y[k] * (t[k + 1] - t[k]) / (y[k + 1] - y[k])
    return float(D / (U * np.mean(np.diff(tc))))


def run(res: int = 36, t_end: float = 200.0, every: int = 20, window: float = 60.0, precision: int = 32,
        smooth_width: float = 1.0) -> dict:
    c = cases.cylinder2d(res=res)
    lam, u, xs = FRINGE
    sim = Simulation(c, precision=precision, body_force=1, fringe_lambda=lam, fringe_u=u, fringe_x=xs)
    ts, cd, cl = [], [], []
    try:
        sim.set_state()
        sim.build_cells()
        t, steps = 0.0, 0
        imp = np.zeros(3)
        t0 = time.perf_counter()
        while t < t_end:
            sim.step(every)
            d = sim.diag()
            steps += every
            # the force averaged over every step of the interval: the change
            # of the body's impulse over the change of the simulated time
            a, b = coefficients((d["body_impulse"] - imp) / (d["time"] - t), c["rho0"], c["U"], 1.0)
            ts.append(0.5 * (t + d["time"]))
            cd.append(a)
            cl.append(b)
            t, imp = d["time"], d["body_impulse"].copy()
        sim.sync()
        wall = time.perf_counter() - t0
    finally:
        sim.close()
    ts, cd, cl = np.array(ts), np.array(cd), np.array(cl)
    late = ts > t_end - window
    cds, cls = smooth(ts, cd, smooth_width), smooth(ts, cl, smooth_width)
    return {"res": res, "D_over_dp_min": 2 * res, "particles": int(c["n"]), "t": float(ts[-1]), "steps": steps,
            "wall_s": wall, "window": [float(t_end - window), float(t_end)], "smoothing_width": smooth_width,
            "C_D_mean": float(cd[late].mean()),
            "C_D_amplitude": float(0.5 * (cds[late].max() - cds[late].min())),
            "C_L_amplitude": float(0.5 * (cls[late].max() - cls[late].min())),
            "St": strouhal(ts[late], cls[late]),
            "paper_table2_present": {"C_D": "1.48 +- 0.015", "C_L": "+-0.405", "St": 0.178, "D_over_dp": 80},
            "history": {"t": ts.tolist(), "C_D": cd.tolist(), "C_L": cl.tolist()}}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--res", type=int, default=36)
    ap.add_argument("--t", type=float, default=200.0)
    ap.add_argument("--every", type=int, default=20)
    ap.add_argument("--window", type=float, default=60.0)
    ap.add_argument("--history", action="store_true", help="print the C_D, C_L history too")
    args = ap.parse_args()
    r = run(args.res, args.t, args.every, args.window)
    if not args.history:
        r.pop("history")
    print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
