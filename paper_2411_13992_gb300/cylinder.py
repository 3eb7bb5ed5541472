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
last ``window`` time units it reports the mean drag and, from the spectrum
of C_L (``shedding``), the Strouhal number St = f D / U and the lift and drag
oscillation amplitudes.  Table 2 of the paper reports C_D = 1.48 +- 0.015,
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


def shedding(t: np.ndarray, cl: np.ndarray, cd: np.ndarray, band=(0.05, 0.5), D=1.0, U=1.0) -> dict:
    """Strouhal number and lift amplitude from a C_L history: the body force
    of a weakly compressible particle method carries acoustic noise (c = 10 U)
    at frequencies far above the shedding frequency, so the history is
    resampled on a uniform grid, the shedding frequency f0 is the largest
    peak of the Hann-windowed spectrum of C_L in ``band`` (in U/D, with a
    Gaussian interpolation between bins), and the lift amplitude is sqrt(2) times the RMS of C_L
    band-passed to [f0/2, 3 f0/2]; the drag oscillates at 2 f0 and is
    band-passed to [3 f0/2, 5 f0/2].  St = f0 D / U."""
    tu = np.linspace(t[0], t[-1], len(t))
    dt = tu[1] - tu[0]
    f = np.fft.rfftfreq(len(tu), dt)
    yl = np.interp(tu, t, cl - cl.mean())
    L = np.fft.rfft(yl)
    Dr = np.fft.rfft(np.interp(tu, t, cd - cd.mean()))
    # the peak from the Hann-windowed spectrum, interpolated on its logarithm
    # (a Gaussian fit through the three bins around the maximum)
    Lw = np.abs(np.fft.rfft(yl * np.hanning(len(yl))))
    sel = np.flatnonzero((f >= band[0]) & (f <= band[1]))
    k = sel[np.argmax(Lw[sel])]
    a, b, c = np.log(Lw[k - 1]), np.log(Lw[k]), np.log(Lw[k + 1])
    f0 = f[k] + 0.5 * (a - c) / (a - 2 * b + c) * (f[1] - f[0])

    def amp(X, lo, hi):
        return float(np.sqrt(2.0) * np.fft.irfft(np.where((f >= lo) & (f <= hi), X, 0), len(tu)).std())

    return {"St": float(f0 * D / U), "C_L_amplitude": amp(L, 0.5 * f0, 1.5 * f0),
            "C_D_amplitude": amp(Dr, 1.5 * f0, 2.5 * f0), "frequency_resolution": float(f[1] - f[0])}


def run(res: int = 36, t_end: float = 200.0, every: int = 20, window: float = 100.0, precision: int = 32) -> dict:
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
    out = {"res": res, "D_over_dp_min": 2 * res, "particles": int(c["n"]), "t": float(ts[-1]), "steps": steps,
           "wall_s": wall, "window": [float(t_end - window), float(t_end)], "C_D_mean": float(cd[late].mean())}
    out.update(shedding(ts[late], cl[late], cd[late]))
    out.update({
        "paper_table2_present": {"C_D": "1.48 +- 0.015", "C_L": "+-0.405", "St": 0.178, "D_over_dp": 80},
        "history": {"t": ts.tolist(), "C_D": cd.tolist(), "C_L": cl.tolist()}})
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--res", type=int, default=36)
    ap.add_argument("--t", type=float, default=200.0)
    ap.add_argument("--every", type=int, default=20)
    ap.add_argument("--window", type=float, default=100.0)
    ap.add_argument("--history", action="store_true", help="print the C_D, C_L history too")
    args = ap.parse_args()
    r = run(args.res, args.t, args.every, args.window)
    if not args.history:
        r.pop("history")
    print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
