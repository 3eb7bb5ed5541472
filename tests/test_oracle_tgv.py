"""Whole-step pins of the oracle on the 2-D Taylor-Green vortex (Sec. 4.1):
the kinetic energy of the exact solution decays like exp(-16 pi^2 nu t).

* Viscosity-dominated (Re = 1, U = 0.01, perfect lattice): the kick-drift-kick
  step must reproduce the decay rate that the SPH viscous operator has on the
  Taylor-Green mode, and that operator must be within 5 % of nu lap.  A
  missing half-kick, a kick with the wrong dt, or a factor error in Eq. 7
  fails this.
* Re = 100 (the paper's case): the limited correction must suppress the
  tensile instability that the uncorrected scheme shows, and the error of the
  decay rate must shrink with resolution.  The tolerance on the Re = 100
  decay rate itself is PARITY UNPINNED (the paper shows its agreement only in
  a figure)."""
import math

import numpy as np
import pytest

from paper_2411_13992_gb300 import cases


def _run(orc, c, nsteps, **kw):
    P = orc.make_params(2, c["lo"], c["L"], c["periodic"], c["rho0"], c["c"], c["eta"], c["h_min"],
                        u_ref=c["u_ref"], **kw)
    s0 = orc.sigma0_for(c, 2)
    fp = orc.force_pass(P, c, c["x"], c["v"], s0)
    st = {"x": c["x"].copy(), "v": c["v"].copy(), "a": fp["a"], "dr": fp["dr"]}
    dt = orc.time_step(P, st["v"], c["kind"])
    ts, ke = [0.0], [0.5 * (c["m"][:, None] * st["v"] ** 2).sum()]
    for _ in range(nsteps):
        st = orc.step(P, c, st, s0, dt)
        ts.append(ts[-1] + dt)
        ke.append(0.5 * (c["m"][:, None] * st["v"] ** 2).sum())
    rate = np.polyfit(np.array(ts), np.log(np.array(ke)), 1)[0]
    return rate / (-16.0 * math.pi ** 2 * c["nu"]), st, P


def test_viscous_decay_matches_operator_and_analytic_rate(orc):
    c = cases.tgv2d(50, U=0.01, Re=1.0, jitter_dp=0.0)
    P = orc.make_params(2, c["lo"], c["L"], c["periodic"], c["rho0"], c["c"], c["eta"], c["h_min"],
                        u_ref=c["u_ref"], riemann_eta=0.0)
    nb = orc.neighbours(P, c["x"], c["h"])
    f = orc.forces(P, c["x"], c["v"], c["h"], c["m"], c["kind"], c["vw"], np.ones(c["n"]), nb)
    lam = (f["a"] * c["v"]).sum() / (c["v"] ** 2).sum() / (-8.0 * math.pi ** 2 * c["nu"])
    assert 0.95 < lam < 1.0, lam                        # SPH Laplacian on the mode vs the exact one
    ratio, _, _ = _run(orc, c, 100)
    assert abs(ratio / lam - 1.0) < 0.01, (ratio, lam)  # time integration adds no decay of its own


def test_limited_correction_suppresses_tensile_instability(orc):
    c = cases.tgv2d(50)
    r_lim, st_lim, _ = _run(orc, c, 150)
    r_none, _, _ = _run(orc, c, 150, tv_mode=0)
    assert r_none > 1.8 and r_lim < 0.6 * r_none, (r_lim, r_none)
    assert (st_lim["chi"] > 0).any()                    # the limiter is active on this flow


@pytest.mark.slow
def test_decay_rate_error_shrinks_with_resolution(orc):
    errs = []
    for n in (25, 50):
        ratio, _, _ = _run(orc, cases.tgv2d(n), 4 * n)
        errs.append(abs(ratio - 1.0))
    assert errs[1] < 0.6 * errs[0], errs


def test_reversed_sum_step_differs_only_by_rounding(orc):
    """The rounding-floor helper takes the same step with neighbour sums in
    the opposite order: identical drift, and fields equal to rounding."""
    c = cases.tgv2d(20)
    P = orc.make_params(2, c["lo"], c["L"], c["periodic"], c["rho0"], c["c"], c["eta"], c["h_min"],
                        u_ref=c["u_ref"])
    s0 = orc.sigma0_for(c, 2)
    fp = orc.force_pass(P, c, c["x"], c["v"], s0)
    st = {"x": c["x"], "v": c["v"], "a": fp["a"], "dr": fp["dr"]}
    dt = orc.time_step(P, c["v"], c["kind"])
    a = orc.step(P, c, st, s0, dt)
    b = orc.step_reversed_sums(P, c, st, s0, dt)
    assert np.array_equal(a["x"], b["x"])
    np.testing.assert_allclose(b["rho"], a["rho"], rtol=1e-14)
    np.testing.assert_allclose(b["v"], a["v"], rtol=0, atol=1e-13)
    assert np.abs(b["a"] - a["a"]).max() < 1e-10 * np.abs(a["a"]).max()
