"""Pins of the oracle's wall branch (reading: a wall neighbour stands in with
rho_j = rho_i, p_j = p_i and its prescribed velocity, and counts in sigma_i
and R_i; the paper gives no wall boundary condition).  The reading is not
fixed by the paper, but it must satisfy these invariants, and a plausible
mistake (walls left out of the density sum or the residual, the wall's
velocity with the wrong sign, walls given rho0 instead of rho_i) breaks one:

* a closed box of fluid at rest on a perfect lattice, with walls at rest, is
  an exact fixed point: rho = rho0, a = 0, R = 0, dr = 0 for every fluid
  particle, also next to the walls and in the corners;
* with the lid moving at U, the fluid (still at rest) next to the lid is
  pulled along +x, the particles farther than 2h from it feel nothing, and
  the pull is exactly linear in U and in eta (no pressure at rest);
* a uniform pressure exerts no force anywhere in the box (the walls, at
  p_j = p_i, complete the kernel support; with walls left out of the sums
  the particles next to them would be pushed)."""
import numpy as np
import pytest

from paper_2411_13992_gb300 import cases


def _box(orc, n=24, U=0.0, eta=None):
    c = cases.cavity2d(n, U=U, jitter_dp=0.0) if U else cases.cavity2d(n, U=1.0, jitter_dp=0.0)
    if not U:
        c["vw"][:] = 0.0
    e = c["eta"] if eta is None else eta
    P = orc.make_params(2, c["lo"], c["L"], c["periodic"], c["rho0"], 10.0, e, c["h_min"])
    s0 = orc.sigma0_for(c, 2)
    return c, P, s0


def test_fluid_at_rest_in_a_walled_box_is_a_fixed_point(orc):
    c, P, s0 = _box(orc)
    out = orc.force_pass(P, c, c["x"], c["v"], s0, mode="brute")
    fl = c["kind"] == 0
    np.testing.assert_allclose(out["rho"][fl], 1.0, rtol=0, atol=1e-14)
    assert np.abs(out["R"][fl]).max() < 1e-13
    assert np.abs(out["dr"][fl]).max() < 1e-13
    assert np.abs(out["a"][fl]).max() < 1e-10


def _lid_pull(orc, U, eta):
    c, P, s0 = _box(orc, U=U, eta=eta)
    P.riemann_eta = 0.0          # the Riemann dissipation is quadratic in U; keep Eq. 7 alone
    out = orc.force_pass(P, c, c["x"], c["v"], s0, mode="brute")
    return c, out["a"]


def test_moving_lid_pulls_the_adjacent_fluid_linearly(orc):
    c, a1 = _lid_pull(orc, 1.0, 0.01)
    _, a2 = _lid_pull(orc, 2.0, 0.01)
    _, a3 = _lid_pull(orc, 1.0, 0.03)
    fl = c["kind"] == 0
    y = c["x"][:, 1]
    near = fl & (y > 1.0 + 0.5 * c["dp"] - 2.0 * c["h_min"] + 1e-9)   # within 2h of the lowest lid row
    far = fl & (y < 1.0 - 2.0 * c["h_min"] - c["dp"]) & (y > 2.0 * c["h_min"] + c["dp"])
    far &= (c["x"][:, 0] > 2.0 * c["h_min"] + c["dp"]) & (c["x"][:, 0] < 1.0 - 2.0 * c["h_min"] - c["dp"])
    assert (a1[near, 0] > 0.0).all()                     # dragged along the lid's motion
    assert np.abs(a1[near, 1]).max() < 1e-12 * a1[near, 0].max()
    assert np.abs(a1[far]).max() < 1e-11                 # beyond the support: rounding noise only
    # (the rest state carries pressure rounding noise of ~1e-12 absolute)
    np.testing.assert_allclose(a2[near, 0], 2.0 * a1[near, 0], rtol=1e-10)
    np.testing.assert_allclose(a3[near, 0], 3.0 * a1[near, 0], rtol=1e-10)


def test_uniform_pressure_exerts_no_force_next_to_walls(orc):
    """With the walls standing in at p_j = p_i, a uniformly compressed fluid at
    rest feels no force anywhere, next to walls and in corners included: the
    walls complete the kernel support, so the pressure term is
    -(2 p / rho_i) R_i with R_i = 0 on the full lattice."""
    c, P, s0 = _box(orc)
    fl = c["kind"] == 0
    rho = np.full(c["n"], 1.0 + 1e-3)                    # p = c^2 (rho - rho0) = 0.1 everywhere
    nb = orc.neighbours(P, c["x"], c["h"], "brute")
    f = orc.forces(P, c["x"], np.zeros_like(c["x"]), c["h"], c["m"], c["kind"], c["vw"], rho, nb)
    scale = 2.0 * 0.1 / 1.001 / c["h_min"]               # 2 p / rho / h: the size of one pair's push
    assert np.abs(f["a"][fl]).max() < 1e-12 * scale
    assert np.abs(f["R"][fl]).max() < 1e-12 / c["h_min"]
