"""Pins of the oracle's dual-criteria time stepping (Sec. 2.4): the Riemann
continuity equation (Eq. 3, first row, with U* of Eq. 5, first row), the two
step-size criteria (Eq. 9-11), the substep loop, and the background-pressure
form of the correction with p0 = alpha rho0 |v|_ad^2 (Eq. 12-13).

Each pin is fixed by mathematics or by values printed in the paper, not by
the oracle's own formulas:
* a rigid rotation does not compress: d rho/dt = 0 for every particle, any
  layout (r^T A r = 0 for antisymmetric A, pair by pair);
* a uniform expansion v = A x compresses at the continuum rate
  d rho/dt = -rho tr A (integration by parts of the kernel gradient), to the
  lattice-moment factor that the pressure-gradient pin also shows (0.97-1);
* with v = 0 the Riemann pressure term of U* is antisymmetric in the pair,
  so sum_i (m_i / rho_i^2) d rho_i/dt = 0, it scales exactly with c, and it
  raises the density at a density minimum;
* Eq. 9-11 by hand (tests/golden/timestep_cases.json);
* position Verlet is exact for a constant acceleration: an isolated particle
  under gravity ends one advection step at x0 + v0 Dt + g Dt^2 / 2;
* pairwise forces conserve momentum over an advection step;
* in the dual scheme Eq. 12 with p0 of Eq. 13 is the displacement
  -alpha CFL_ad^2 h^2 (rho0 / rho_i) R_i (alpha = 7, tests/golden);
* the viscosity-dominated Taylor-Green vortex decays at the SPH viscous
  operator's rate, within the first-order error of holding the viscous
  force over an advection step (the forward-Euler bound lambda Dt)."""
import json
import math
import os

import numpy as np
import pytest

from paper_2411_13992_gb300 import cases

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _block(orc, dim, n, periodic, jitter=0.0, c0=10.0, eta=0.0, **kw):
    c = cases.lattice_block(dim, n, dp=1.0, periodic=periodic, jitter_dp=jitter, seed=7)
    P = orc.make_params(dim, c["lo"], c["L"], c["periodic"], 1.0, c0, eta, c["h_min"], **kw)
    return c, P


def _interior(c, dim, margin):
    ok = np.ones(c["n"], bool)
    for d in range(dim):
        ok &= (c["x"][:, d] > margin) & (c["x"][:, d] < c["L"][d] - margin)
    return ok


@pytest.mark.parametrize("dim,n", [(2, 16), (3, 8)])
def test_rotation_does_not_compress(orc, dim, n):
    c, P = _block(orc, dim, n, periodic=False, jitter=0.15)
    A = np.zeros((3, 3))
    A[0, 1], A[1, 0] = 0.3, -0.3
    if dim == 3:
        A[1, 2], A[2, 1] = -0.2, 0.2
    v = c["x"] @ A.T
    nb = orc.neighbours(P, c["x"], c["h"], "brute")
    drho = orc.continuity(P, c["x"], v, c["h"], c["m"], c["kind"], c["vw"], np.ones(c["n"]), nb)
    assert np.abs(drho).max() < 1e-13 * np.abs(v).max()


@pytest.mark.parametrize("dim,n", [(2, 30), (3, 14)])
def test_expansion_compresses_at_minus_rho_div_v(orc, dim, n):
    c, P = _block(orc, dim, n, periodic=False)
    A = np.diag([1.0e-3, 2.0e-3, 1.5e-3 if dim == 3 else 0.0])
    v = c["x"] @ A.T
    nb = orc.neighbours(P, c["x"], c["h"], "brute")
    drho = orc.continuity(P, c["x"], v, c["h"], c["m"], c["kind"], c["vw"], np.ones(c["n"]), nb)
    inner = _interior(c, dim, 3.5)
    ratio = drho[inner] / (-1.0 * np.trace(A))
    assert 0.97 < ratio.mean() < 1.0, ratio.mean()
    assert ratio.std() < 1e-6


def _pressure_term(orc, c0):
    c, P = _block(orc, 2, 16, periodic=True, jitter=0.1, c0=c0)
    rng = np.random.default_rng(3)
    rho = 1.0 + 1.0e-3 * rng.standard_normal(c["n"])
    nb = orc.neighbours(P, c["x"], c["h"])
    drho = orc.continuity(P, c["x"], np.zeros_like(c["x"]), c["h"], c["m"], c["kind"], c["vw"], rho, nb)
    return c, rho, drho


def test_pressure_term_of_ustar_is_antisymmetric_scales_with_c_and_smooths(orc):
    c, rho, d1 = _pressure_term(orc, 10.0)
    _, _, d2 = _pressure_term(orc, 20.0)
    w = c["m"] / rho ** 2
    assert abs((w * d1).sum()) < 1e-13 * (w * np.abs(d1)).sum()
    np.testing.assert_allclose(d2, 2.0 * d1, rtol=1e-12, atol=1e-15 * np.abs(d1).max())
    assert d1[np.argmin(rho)] > 0.0 and d1[np.argmax(rho)] < 0.0
    assert np.abs(d1).max() > 0.0


def test_interface_velocity_values(orc):
    """Eq. 5 (first row) with rho_bar c = 20: U* = (U_l + U_r)/2 + (p_l - p_r)/40."""
    P = orc.make_params(2, (0, 0, 0), (1, 1, 1), (0, 0, 0), 1.0, 10.0, 0.0, 0.1)
    assert orc.riemann_ustar(P, 4.0, 2.0, 2.0, 1.0, 0.5) == pytest.approx(0.75 + 0.05, rel=1e-15)
    assert orc.riemann_ustar(P, 2.0, 2.0, 2.0, -1.0, 1.0) == 0.0


def test_advection_and_acoustic_step_hand_values(orc):
    for case in _gold("timestep_cases.json")["cases"]:
        P = orc.make_params(2, (0, 0, 0), (1, 1, 1), (1, 1, 0), 1.0, case["c"], case["nu"], case["h"],
                            u_ref=case["u_ref"])
        v = np.zeros((3, 3))
        v[1, 0], v[1, 1] = 0.6 * case["vmax"], 0.8 * case["vmax"]
        kind = np.zeros(3, np.int8)
        dt_ad, vad = orc.advection_step(P, v, kind)
        assert dt_ad == pytest.approx(case["dt_ad"], rel=1e-12), case["why"]
        assert vad == pytest.approx(0.25 * case["h"] / case["dt_ad"], rel=1e-12)
        assert orc.acoustic_step(P, v, kind) == pytest.approx(case["dt_ac"], rel=1e-12), case["why"]


def test_isolated_particles_under_gravity_follow_the_parabola(orc):
    """Particles 3 h apart have no neighbour but themselves: every substep is
    drift-kick-drift under g alone, exact for a constant acceleration."""
    n = 4
    x = np.zeros((n, 3))
    x[:, 0] = 1.0 + 3.9 * np.arange(n)
    x[:, 1] = 5.0
    v = np.zeros((n, 3))
    v[:, 0] = [0.1, -0.2, 0.0, 0.05]
    v[:, 1] = [0.3, 0.0, -0.1, 0.2]
    g = (0.0, -0.5, 0.0)
    case = {"n": n, "h": np.full(n, 1.3), "m": np.ones(n), "kind": np.zeros(n, np.int8), "vw": np.zeros((n, 3))}
    P = orc.make_params(2, (0, 0, 0), (20.0, 10.0, 1.0), (0, 0, 0), 1.0, 10.0, 0.0, 1.3, g=g, u_ref=0.4)
    s0 = np.full(n, orc.lattice_sum(2, 1.3))
    out = orc.dual_step(P, case, {"x": x, "v": v, "drho": np.zeros(n)}, s0, mode="brute")
    Dt = out["Dt"]
    assert Dt == pytest.approx(0.25 * 1.3 / 0.4, rel=1e-15)       # |v|max <= u_ref here
    gv = np.array(g)
    np.testing.assert_allclose(out["x"], x + v * Dt + 0.5 * gv * Dt ** 2, rtol=0, atol=1e-13)
    np.testing.assert_allclose(out["v"], v + gv * Dt, rtol=0, atol=1e-14)
    assert np.abs(out["drho"]).max() == 0.0
    vmax_end = np.sqrt((out["v"] ** 2).sum(1)).max()
    assert Dt / (0.6 * 1.3 / 10.0) <= out["substeps"] <= Dt / (0.6 * 1.3 / (10.0 + vmax_end)) + 1


def test_advection_step_conserves_momentum(orc):
    c = cases.tgv2d(16, jitter_dp=0.1, seed=5)
    P = orc.make_params(2, c["lo"], c["L"], c["periodic"], c["rho0"], c["c"], c["eta"], c["h_min"],
                        u_ref=c["u_ref"])
    s0 = orc.sigma0_for(c, 2)
    st = {"x": c["x"], "v": c["v"], "drho": np.zeros(c["n"])}
    for _ in range(3):
        out = orc.dual_step(P, c, st, s0)
        st = out
        assert out["substeps"] >= 4
    p0 = (c["m"][:, None] * c["v"]).sum(0)
    p1 = (c["m"][:, None] * out["v"]).sum(0)
    assert np.abs(p1 - p0).max() < 1e-14 * (c["m"][:, None] * np.abs(c["v"])).sum()


def test_background_form_is_alpha_cfl_squared_displacement(orc):
    alpha = _gold("paper_constants.json")["bg_alpha"]["value"]
    c = cases.tgv2d(16, jitter_dp=0.2, seed=9)
    P = orc.make_params(2, c["lo"], c["L"], c["periodic"], c["rho0"], c["c"], c["eta"], c["h_min"],
                        u_ref=c["u_ref"], tv_mode=orc.TV_BACKGROUND)
    s0 = orc.sigma0_for(c, 2)
    out = orc.dual_step(P, c, {"x": c["x"], "v": c["v"], "drho": np.zeros(c["n"])}, s0)
    # the density of the correction is the one summed at the start of the step
    nb = orc.neighbours(P, c["x"], c["h"])
    rho0_step, _ = orc.density(P, c["x"], c["h"], c["kind"], s0, nb)
    expect = -alpha * P.cfl_ad ** 2 * c["h_min"] ** 2 * (c["rho0"] / rho0_step)[:, None] * out["R"]
    np.testing.assert_allclose(out["dr"], expect, rtol=0, atol=1e-14 * np.abs(expect).max())
    assert np.abs(expect).max() > 0.0


def test_viscous_taylor_green_decays_at_the_operator_rate(orc):
    c = cases.tgv2d(50, U=0.01, Re=1.0, jitter_dp=0.0)
    P = orc.make_params(2, c["lo"], c["L"], c["periodic"], c["rho0"], c["c"], c["eta"], c["h_min"],
                        u_ref=c["u_ref"], riemann_eta=0.0)
    nb = orc.neighbours(P, c["x"], c["h"])
    f = orc.forces(P, c["x"], c["v"], c["h"], c["m"], c["kind"], c["vw"], np.ones(c["n"]), nb)
    lam = (f["a"] * c["v"]).sum() / (c["v"] ** 2).sum() / (-8.0 * math.pi ** 2 * c["nu"])
    s0 = orc.sigma0_for(c, 2)
    st = {"x": c["x"], "v": c["v"], "drho": np.zeros(c["n"])}
    ts, ke = [0.0], [0.5 * (c["m"][:, None] * c["v"] ** 2).sum()]
    for _ in range(20):
        st = orc.dual_step(P, c, st, s0)
        ts.append(ts[-1] + st["Dt"])
        ke.append(0.5 * (c["m"][:, None] * st["v"] ** 2).sum())
    rate = np.polyfit(np.array(ts), np.log(np.array(ke)), 1)[0] / (-16.0 * math.pi ** 2 * c["nu"])
    lam_v = 8.0 * math.pi ** 2 * c["nu"] * lam         # velocity decay rate of the SPH operator
    assert abs(rate / lam - 1.0) < lam_v * st["Dt"], (rate, lam, lam_v * st["Dt"])
