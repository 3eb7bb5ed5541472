"""Pins of the Riemann interface pressure (Eq. 5-6), the limiter (Eq. 15),
the time-step criteria (Eq. 9-11) and the paper's constants, from values the
paper prints or that follow from its formulas by hand (tests/golden)."""
import json
import math
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _P(orc, **kw):
    return orc.make_params(2, (0, 0, 0), (1, 1, 1), (0, 0, 0), 1.0, 10.0, 0.0, 0.1, **kw)


def test_oracle_defaults_are_the_papers_constants(orc):
    g = _gold("paper_constants.json")
    P = _P(orc)
    for k in ("riemann_eta", "tv_C", "tv_thresh", "tv_xi", "cfl_ad", "cfl_ac"):
        assert getattr(P, k) == g[k]["value"], k
    from paper_2411_13992_gb300 import cases
    assert cases.H_OVER_DP == g["h_over_dp"]["value"]
    c = cases.tgv2d(10)
    assert c["c"] == g["c_over_umax"]["value"] * c["U"]


def test_riemann_limiter_values(orc):
    """Eq. 6 with eta = 3: beta = min(3 max(dU/c, 0), 1)."""
    P = _P(orc)
    assert orc.riemann_beta(P, 0.5, 0.0) == pytest.approx(0.15, rel=1e-15)      # dU/c = 0.05
    assert orc.riemann_beta(P, 1.0, -1.0) == pytest.approx(0.6, rel=1e-15)      # dU/c = 0.2
    assert orc.riemann_beta(P, 3.0, -1.0) == 1.0                                # dU/c = 0.4 > 1/3
    assert orc.riemann_beta(P, -1.0, 1.0) == 0.0                                # separating
    # beta = 1 turns Eq. 5 into the linearised solver of Eq. 4
    assert orc.riemann_pstar(P, 2.0, 4.0, 1.5, 5.0, 0.0) == pytest.approx(3.0 + 0.5 * 1.5 * 10.0 * 5.0)


def _pair_force(orc, u, eps=0.0):
    """Two particles on the x axis, j to the right of i, closing speed u
    (u < 0: separating), both at density 1 + eps."""
    from paper_2411_13992_gb300 import cases
    P = orc.make_params(2, (0, 0, 0), (10, 10, 1), (0, 0, 0), 1.0, 10.0, 0.0, 1.3)
    x = np.array([[5.0, 5.0, 0.0], [6.0, 5.0, 0.0]])
    v = np.array([[0.5 * u, 0.0, 0.0], [-0.5 * u, 0.0, 0.0]])
    h, m, kind = np.full(2, 1.3), np.ones(2), np.zeros(2, np.int8)
    nb = orc.neighbours(P, x, h, "brute")
    f = orc.forces(P, x, v, h, m, kind, np.zeros((2, 3)), np.full(2, 1.0 + eps), nb)
    return f["a"]


def test_pair_force_sign_and_dissipation_scaling(orc):
    # positive pressure repels: i is pushed to -x, j to +x
    a = _pair_force(orc, 0.0, eps=1e-3)
    assert a[0, 0] < 0 < a[1, 0]
    assert a[0, 0] == pytest.approx(-a[1, 0], rel=1e-14)
    # no pressure: only the Riemann dissipation acts, ~ beta * u
    f = lambda u: _pair_force(orc, u)[0, 0]
    assert f(0.0) == 0.0
    assert f(-0.5) == 0.0 and f(-8.0) == 0.0                 # separating: beta = 0
    assert f(0.5) < 0.0                                     # approaching: repulsive
    assert f(1.0) / f(0.5) == pytest.approx(4.0, rel=1e-12)  # beta ~ u  -> force ~ u^2
    assert f(8.0) / f(4.0) == pytest.approx(2.0, rel=1e-12)  # beta = 1  -> force ~ u


def test_transport_limiter_values(orc):
    """Eq. 15 with C = 1e3, threshold 5e-4 (strict)."""
    P = _P(orc)
    assert orc.tv_limiter(P, 0.0) == 0.0
    assert orc.tv_limiter(P, 4.9e-4) == 0.0
    assert orc.tv_limiter(P, 5.0e-4) == 0.0
    assert orc.tv_limiter(P, 6.0e-4) == pytest.approx(0.6, rel=1e-14)
    assert orc.tv_limiter(P, 9.0e-4) == pytest.approx(0.9, rel=1e-14)
    assert orc.tv_limiter(P, 2.0e-3) == 1.0
    assert orc.tv_limiter(_P(orc, tv_mode=0), 1.0) == 0.0
    assert orc.tv_limiter(_P(orc, tv_mode=2), 0.0) == 1.0


def test_time_step_hand_values(orc):
    for case in _gold("timestep_cases.json")["cases"]:
        P = orc.make_params(2, (0, 0, 0), (1, 1, 1), (1, 1, 0), 1.0, case["c"], case["nu"], case["h"],
                            u_ref=case["u_ref"])
        v = np.zeros((3, 3))
        v[1, 0] = case["vmax"] * 0.6
        v[1, 1] = case["vmax"] * 0.8
        v[2, 0] = 0.3 * case["vmax"]
        dt = orc.time_step(P, v, np.zeros(3, np.int8))
        assert dt == pytest.approx(case["dt"], rel=1e-12), case["why"]


def test_background_pressure_mode_equals_uniform_pressure_force(orc):
    """Eq. 12: the transport correction of Adami's formulation is the
    acceleration of a uniform background pressure p0 = rho0 c^2, applied as
    the displacement dt^2/2 a_bg in the drift.  With every particle at rest
    and rho = 2 rho0 (so the EOS gives p = rho0 c^2 = p0 everywhere), the
    pressure force of Eq. 3 is exactly that acceleration."""
    from paper_2411_13992_gb300 import cases
    c = cases.lattice_block(2, 12, dp=0.1, jitter_dp=0.2, seed=4)
    P = orc.make_params(2, c["lo"], c["L"], c["periodic"], 1.0, 10.0, 0.0, c["h_min"], tv_mode=3)
    P.dt_tv = 1.7e-3
    nb = orc.neighbours(P, c["x"], c["h"])
    rho = np.full(c["n"], 2.0)
    f = orc.forces(P, c["x"], np.zeros((c["n"], 3)), c["h"], c["m"], c["kind"], c["vw"], rho, nb)
    np.testing.assert_allclose(f["dr"], 0.5 * P.dt_tv ** 2 * f["a"], rtol=0,
                               atol=1e-13 * np.abs(0.5 * P.dt_tv ** 2 * f["a"]).max())
    assert np.abs(f["dr"]).max() > 0
