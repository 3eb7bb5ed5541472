"""Lid-driven cavity at Re = 1000 (Sec. 4.2), self-convergence: the case
runner (paper_2411_13992_gb300.cavity, the dual-criteria integrator in FP32)
at dp = 1/50, 1/100 and 1/200, the centre-line profiles u(0.5, y) and
v(x, 0.5) averaged over t in [12, 20].  The paper compares the profiles with
Ghia et al.'s data, which are not in the repository; what is checked here is
self-convergence: the RMS difference between successive resolutions'
profiles shrinks as dp halves, and the extremes of the averaged profiles move
monotonically with resolution.  (The weakly compressible flow at Re = 1000
fluctuates, and its instantaneous extremes move by a few percent under FP32
rounding changes alone; the time average is what converges.  Measured ratio
of the two differences 0.60-0.63 over two rounding variants of the density
pass and two averaging windows.)"""
import numpy as np
import pytest

from paper_2411_13992_gb300 import cavity

pytestmark = pytest.mark.gpu


def test_cavity_re1000_averaged_profiles_converge():
    runs = {n: cavity.run(n, 20.0, average_from=12.0) for n in (50, 100, 200)}
    prof = {n: np.concatenate([r["u_on_x_half"], r["v_on_y_half"]]) for n, r in runs.items()}
    d1 = np.sqrt(np.mean((prof[100] - prof[50]) ** 2))
    d2 = np.sqrt(np.mean((prof[200] - prof[100]) ** 2))
    for n, r in runs.items():
        print(n, "u_min %.4f v_max %.4f v_min %.4f, %d samples, %d advection steps, %.1f s"
              % (r["u_min"], r["v_max"], r["v_min"], r["samples"], r["advection_steps"], r["wall_s"]))
        assert abs(r["t"] - 20.0) < 0.01 and r["samples"] >= 15
    print("RMS differences: 50/100 %.4f, 100/200 %.4f" % (d1, d2))
    assert d2 < 0.8 * d1
    e = {k: [runs[n][k] for n in (50, 100, 200)] for k in ("u_min", "v_max", "v_min")}
    assert e["u_min"][0] > e["u_min"][1] > e["u_min"][2], e
    assert e["v_max"][0] < e["v_max"][1] < e["v_max"][2], e
    assert e["v_min"][0] > e["v_min"][1] > e["v_min"][2], e
    # the primary vortex is established: extremes of the size the finer runs
    # reach at t = 60 (u_min ~ -0.35, v in [-0.49, 0.34])
    assert runs[200]["u_min"] < -0.25 and runs[200]["v_max"] > 0.22 and runs[200]["v_min"] < -0.38
