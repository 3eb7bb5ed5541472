"""The overcorrection case of Sec. 3 with the dual-criteria integrator: the
2-D Taylor-Green vortex at dp = 1/200, Re = 100, to t = 5 (40,000 particles,
about 4,700 advection steps per run, FP32).

What the paper states and these GPU runs reproduce:
* the unlimited correction (Eq. 14) overcorrects: late in the decay its
  transport speed max|v + dr/Dt| exceeds the fluid speed max|v| and the
  kinetic energy decays more slowly than the analytic exp(-16 pi^2 t / Re);
* the background-pressure form (Eq. 12 with p0 of Eq. 13) does the same;
* without a correction the tensile instability drains the kinetic energy;
* the limiter (Eq. 15) corrects only particles above its threshold.
The paper's further claim, that the limited correction (Eq. 16) follows the
analytic decay, is not reproduced with Eq. 15 as printed (the limited run
decays faster than the analytic rate); that is recorded, not asserted."""
import math

import numpy as np
import pytest
import torch

import paper_2411_13992_gb300 as sph
from paper_2411_13992_gb300 import cases

pytestmark = pytest.mark.gpu


def _run(tv_mode, T=5.0, n=200):
    c = cases.tgv2d(n)
    sim = sph.Simulation(c, precision=32, tv_mode=tv_mode, integrator=sph.INT_DUAL)
    try:
        sim.set_state()
        sim.build_cells()
        ke0 = sim.diag()["ke"]
        t, rows = 0.0, []
        while t < T:
            sim.step(10)
            d = sim.diag()
            t += 10 * d["dt"]
            rows.append((t, d["vt_max"] / d["vmax"], d["ke"] / ke0 / math.exp(-16 * math.pi ** 2 * c["nu"] * t),
                         d["n_chi"]))
        assert sim.sync() is None
    finally:
        sim.close()
    return c, np.array(rows)


@pytest.fixture(scope="module")
def runs():
    assert torch.cuda.is_available()
    return {name: _run(mode) for name, mode in (("unlimited", sph.TV_UNLIMITED), ("limited", sph.TV_LIMITED),
                                                 ("background", sph.TV_BACKGROUND), ("none", sph.TV_OFF))}


def test_unlimited_correction_overcorrects_late_in_the_decay(runs):
    c, r = runs["unlimited"]
    late = r[:, 0] > 3.0
    print("unlimited: max vt/v %.3f, KE/analytic at t=5 %.3f" % (r[late, 1].max(), r[-1, 2]))
    assert r[late, 1].max() > 1.0            # transport speed above the fluid speed
    assert r[-1, 2] > 1.2                    # less decay than the analytic solution
    assert (r[:, 3] == c["n"]).all()         # chi = 1 everywhere


def test_background_pressure_form_overcorrects_too(runs):
    _, r = runs["background"]
    print("background: KE/analytic at t=5 %.3f" % r[-1, 2])
    assert r[-1, 2] > 1.2


def test_no_correction_loses_energy_and_the_limiter_is_selective(runs):
    c, rn = runs["none"]
    _, rl = runs["limited"]
    _, ru = runs["unlimited"]
    print("KE/analytic at t=0.5, 2, 5: none %s limited %s unlimited %s" % tuple(
        np.round(np.interp([0.5, 2.0, 5.0], r[:, 0], r[:, 2]), 3) for r in (rn, rl, ru)))
    assert rn[-1, 2] < 0.1 and np.interp(0.5, rn[:, 0], rn[:, 2]) < 0.6
    after = rl[:, 0] > 0.3                  # (identical at first: the limiter corrects nothing yet)
    assert (rl[after, 2] > np.interp(rl[after, 0], rn[:, 0], rn[:, 2])).all()    # limited loses less than none
    assert rl[:, 3].max() < 0.35 * c["n"]          # most particles uncorrected (measured <= 22 %)
