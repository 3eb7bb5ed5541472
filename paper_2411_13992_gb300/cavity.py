"""Lid-driven cavity at Re = 1000 (Sec. 4.2): the case runner and its
centre-line profiles.

``run(n, t_end)`` steps ``cases.cavity2d(n, U=1, Re=1000)`` -- n x n fluid
particles in the unit square, three layers of lattice wall particles, the
top layers moving with the lid -- with the dual-criteria integrator
(Sec. 2.4) of the library, in FP32, to the time ``t_end``, and returns the
velocity profiles on the two centre lines: u(0.5, y) and v(x, 0.5) at
``points`` interior stations.  The profiles are sampled from the particles
by a Shepard-normalised kernel sum (Wendland C2 at the particles' h, fluid
particles only): q(p) = sum_j q_j V_j W(|p - x_j|) / sum_j V_j W(|p - x_j|).

The paper compares these profiles with the data of Ghia et al., which are
not part of this repository; what can be measured here is self-convergence:
the extremes of the profiles as the resolution dp = 1/n is refined.

    python -m paper_2411_13992_gb300.cavity --n 50 100 200 --t 60

prints one JSON line per resolution (the extremes, the simulated time, the
advection steps and the wall time).
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import INT_DUAL, Simulation, cases

RE = 1000.0


def stations(points: int) -> np.ndarray:
    """Interior stations (k + 1/2) / points, k = 0 .. points - 1."""
    return (np.arange(points) + 0.5) / points


def _wendland2d(r: np.ndarray, h: np.ndarray) -> np.ndarray:
    q = r / h
    w = 7.0 / (4.0 * math.pi * h * h) * (1.0 - 0.5 * q) ** 4 * (2.0 * q + 1.0)
    return np.where(q < 2.0, w, 0.0)


def sample(x: np.ndarray, vel: np.ndarray, h: np.ndarray, vol: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """Shepard-normalised kernel sum of the velocity at the points pts [k][2]."""
    out = np.zeros((len(pts), 2))
    for k, p in enumerate(pts):
        r = np.hypot(x[:, 0] - p[0], x[:, 1] - p[1])
        near = r < 2.0 * h
        w = _wendland2d(r[near], h[near]) * vol[near]
        out[k] = (w[:, None] * vel[near, :2]).sum(axis=0) / w.sum()
    return out


def _profiles(c, st, points):
    fl = c["kind"] == 0
    x, vel, h = st["x"][fl], st["v"][fl], c["h"][fl]
    vol = c["m"][fl] / st["rho"][fl]
    s = stations(points)
    u_line = sample(x, vel, h, vol, np.stack([np.full(points, 0.5), s], axis=1))[:, 0]
    v_line = sample(x, vel, h, vol, np.stack([s, np.full(points, 0.5)], axis=1))[:, 1]
    return u_line, v_line


def run(n: int, t_end: float, points: int = 37, precision: int = 32, average_from: float | None = None,
        sample_dt: float = 0.5, **params) -> dict:
    """Step the Re = 1000 cavity at dp = 1/n to t_end; centre-line profiles
    at t_end, or averaged over samples every sample_dt from average_from to
    t_end (the weakly compressible flow at Re = 1000 fluctuates: the
    instantaneous extremes move by a few percent from one time to the next).
    Extra keyword arguments are sph_params fields."""
    c = cases.cavity2d(n, U=1.0, Re=RE)
    sim = Simulation(c, precision=precision, integrator=INT_DUAL, **params)
    u_acc, v_acc, nsamp = 0.0, 0.0, 0
    try:
        sim.set_state()
        sim.build_cells()
        t, steps = 0.0, 0
        t_next = average_from
        t0 = time.perf_counter()
        while t < t_end:
            sim.step(1)
            t += sim.diag()["dt"]
            steps += 1
            if t_next is not None and t >= t_next and t < t_end:
                u_line, v_line = _profiles(c, sim.get_state(), points)
                u_acc, v_acc, nsamp = u_acc + u_line, v_acc + v_line, nsamp + 1
                t_next += sample_dt
        sim.sync()
        wall = time.perf_counter() - t0
        u_line, v_line = _profiles(c, sim.get_state(), points)
        if t_next is not None:
            u_line, v_line = (u_acc + u_line) / (nsamp + 1), (v_acc + v_line) / (nsamp + 1)
            nsamp += 1
    finally:
        sim.close()
    return {"n": n, "dp": 1.0 / n, "t": t, "advection_steps": steps, "wall_s": wall,
            "samples": max(nsamp, 1), "average_from": average_from,
            "u_min": float(u_line.min()), "v_max": float(v_line.max()), "v_min": float(v_line.min()),
            "u_on_x_half": u_line.tolist(), "v_on_y_half": v_line.tolist(), "stations": stations(points).tolist()}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--n", type=int, nargs="+", default=[50, 100, 200])
    ap.add_argument("--t", type=float, default=60.0)
    ap.add_argument("--points", type=int, default=37)
    ap.add_argument("--average-from", type=float, default=None,
                    help="average the profiles over samples from this time to --t")
    ap.add_argument("--profiles", action="store_true", help="print the sampled profiles too")
    args = ap.parse_args()
    for n in args.n:
        r = run(n, args.t, args.points, average_from=args.average_from)
        if not args.profiles:
            for k in ("u_on_x_half", "v_on_y_half", "stations"):
                r.pop(k)
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
