"""Lid-driven cavity at Re = 1000 (Sec. 4.2), self-convergence: the case
runner (paper_2411_13992_gb300.cavity, the dual-criteria integrator in FP32)
at dp = 1/50, 1/100 and 1/200 to t = 20.  The paper compares the centre-line
profiles with Ghia et al.'s data, which are not in the repository; what is
checked here is that the extremes of u(0.5, y) and v(x, 0.5) converge as the
resolution is refined: the differences between successive resolutions
shrink, and the extremes of v move monotonically toward the finest run."""
import pytest

from paper_2411_13992_gb300 import cavity

pytestmark = pytest.mark.gpu


def test_cavity_re1000_centre_line_extremes_converge():
    runs = {n: cavity.run(n, 20.0) for n in (50, 100, 200)}
    for n, r in runs.items():
        print(n, "u_min %.4f v_max %.4f v_min %.4f (%d advection steps, %.1f s)"
              % (r["u_min"], r["v_max"], r["v_min"], r["advection_steps"], r["wall_s"]))
        assert abs(r["t"] - 20.0) < 0.01
    for key in ("u_min", "v_max", "v_min"):
        e = [runs[n][key] for n in (50, 100, 200)]
        assert abs(e[2] - e[1]) < abs(e[1] - e[0]), (key, e)
    for key, sign in (("v_max", 1.0), ("v_min", -1.0)):
        e = [runs[n][key] for n in (50, 100, 200)]
        assert sign * (e[1] - e[0]) > 0.0 and sign * (e[2] - e[1]) > 0.0, (key, e)
    # the primary vortex is established: the extremes are of the size the
    # finer runs reach at t = 60 (|u_min| ~ 0.35, v in [-0.49, 0.34])
    assert runs[200]["u_min"] < -0.25 and runs[200]["v_max"] > 0.25 and runs[200]["v_min"] < -0.4
