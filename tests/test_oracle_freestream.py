"""Pins of the oracle's free-stream forcing and body force (flow past the
cylinder, Sec. 4.4 and Eq. 18).

The paper names a free-stream boundary condition for the cylinder case but
does not give it; the build stands the fringe-region forcing of Nordstrom,
Nordin & Henningson (1999) in for it: lambda(x) (U_inf - v) added to the
momentum equation in a region of a periodic box, lambda(x) = lambda_max
[S((x - x0)/d_rise) - S((x - x1)/d_fall + 1)] with the smooth step
S(t) = 1 / (1 + exp(1/(t - 1) + 1/t)).  The pins use what that definition
fixes (the step's symmetry S(t) + S(1 - t) = 1, the plateau, the support,
smoothness, the closed-form acceleration of an isolated particle) and the
momentum balance that defines the force on the walls."""
import numpy as np
import pytest

from paper_2411_13992_gb300 import cases

LAM, U, XS = 5.0, (1.0, 0.0, 0.0), (24.0, 29.0, 2.0, 1.0)


def _params(orc, dim=2, lo=(0, 0, 0), L=(30.0, 16.0, 1.0), periodic=(1, 1, 0), eta=0.01, h_min=0.05, **kw):
    return orc.make_params(dim, lo, L, periodic, 1.0, 10.0, eta, h_min, fringe=(LAM, U, XS), **kw)


def test_fringe_rate_support_plateau_and_symmetric_step(orc):
    P = _params(orc)
    x0, x1, rise, fall = XS
    for x in (0.0, 10.0, x0 - 1e-9, x0, x1, x1 + 0.3, 30.0):
        assert orc.fringe_rate(P, x) == 0.0, x
    for x in np.linspace(x0 + rise, x1 - fall, 7):
        assert orc.fringe_rate(P, x) == LAM
    assert orc.fringe_rate(P, x0 + 0.5 * rise) == pytest.approx(0.5 * LAM, rel=1e-15)
    assert orc.fringe_rate(P, x1 - 0.5 * fall) == pytest.approx(0.5 * LAM, rel=1e-15)
    for t in np.linspace(0.05, 0.95, 19):                # S(t) + S(1 - t) = 1 on the rise and the fall
        up = orc.fringe_rate(P, x0 + t * rise) + orc.fringe_rate(P, x0 + (1 - t) * rise)
        down = orc.fringe_rate(P, x1 - fall + t * fall) + orc.fringe_rate(P, x1 - fall + (1 - t) * fall)
        assert up == pytest.approx(LAM, rel=1e-14) and down == pytest.approx(LAM, rel=1e-14)
    # monotone rise, and flat (all derivatives vanish) at both ends of the rise
    xs = np.linspace(x0, x0 + rise, 201)
    lam = np.array([orc.fringe_rate(P, x) for x in xs])
    assert np.all(np.diff(lam) >= 0.0)
    e = 1e-3 * rise
    for end in (x0 + e, x0 + rise - e):
        slope = (orc.fringe_rate(P, end + 0.5 * e) - orc.fringe_rate(P, end - 0.5 * e)) / e
        assert abs(slope) < 1e-100 + 1e-6 * LAM / rise
    off = orc.make_params(2, (0, 0, 0), (30.0, 16.0, 1.0), (1, 1, 0), 1.0, 10.0, 0.01, 0.05)
    assert orc.fringe_rate(off, 26.0) == 0.0             # no forcing unless switched on


def test_isolated_particle_gets_the_closed_form_forcing(orc):
    """No neighbours: a = g + lambda(x) (U_inf - v) exactly."""
    g = (0.0, -0.3, 0.0)
    P = _params(orc, g=g)
    x = np.array([[26.0, 8.0, 0.0], [24.7, 3.0, 0.0], [12.0, 8.0, 0.0]])
    v = np.array([[0.2, 0.5, 0.0], [-1.0, 0.25, 0.0], [0.3, 0.1, 0.0]])
    h = np.full(3, 0.05)
    m = np.full(3, 0.01)
    kind = np.zeros(3, np.int8)
    nb = orc.neighbours(P, x, h, "brute")
    f = orc.forces(P, x, v, h, m, kind, np.zeros((3, 3)), np.ones(3), nb)
    for i in range(3):
        lam = orc.fringe_rate(P, x[i, 0])
        want = np.array(g) + lam * (np.array(U) - v[i])
        want[2] = 0.0
        np.testing.assert_allclose(f["a"][i], want, rtol=0, atol=1e-15)
    assert orc.fringe_rate(P, x[2, 0]) == 0.0 and orc.fringe_rate(P, x[0, 0]) == LAM


def test_uniform_free_stream_on_a_lattice_is_left_alone(orc):
    """A periodic perfect lattice moving with the free stream feels no force
    (the pair sums vanish and the forcing is zero at v = U_inf)."""
    c = cases.lattice_block(2, 24, dp=0.5)
    P = orc.make_params(2, c["lo"], c["L"], c["periodic"], 1.0, 10.0, 0.01, c["h_min"],
                        fringe=(LAM, U, (3.0, 9.0, 2.0, 1.0)))
    v = np.tile(np.array(U), (c["n"], 1))
    s0 = orc.sigma0_for(c, 2)
    out = orc.force_pass(P, c, c["x"], v, s0, mode="brute")
    assert np.abs(out["a"]).max() < 1e-11


def _cylinder():
    return cases.cylinder2d(D=1.0, res=12, box=(6.0, 3.0), center=(2.0, 1.5), refine=(1.0, 4.5, 0.5, 2.5),
                            band_dp=2.0, U=1.0)


def test_wall_force_is_the_momentum_the_walls_take_from_the_fluid(orc):
    """Fluid-fluid pair terms cancel pairwise, so the force on the walls is
    minus the fluid's momentum rate less gravity and the free-stream forcing:
    F_w = -(sum_i m_i a_i - M g - sum_i m_i lambda_i (U_inf - v_i))."""
    g = (0.0, -0.2, 0.0)
    for c, fr in ((_cylinder(), (LAM, U, (4.5, 5.8, 0.6, 0.4))), (cases.cavity2d(20, U=1.0), None)):
        P = orc.make_params(2, c["lo"], c["L"], c["periodic"], c["rho0"], c["c"], c["eta"], c["h_min"],
                            g=g, fringe=fr)
        fl = c["kind"] == 0
        v = c["v"].copy()
        v[fl, 1] += 0.1 * np.sin(3.0 * c["x"][fl, 0])        # a non-uniform flow
        s0 = orc.sigma0_for(c, 2)
        nb = orc.neighbours(P, c["x"], c["h"], "cells")
        rho, _ = orc.density(P, c["x"], c["h"], c["kind"], s0, nb)
        f = orc.forces(P, c["x"], v, c["h"], c["m"], c["kind"], c["vw"], rho, nb)
        F = orc.wall_force(P, c["x"], v, c["h"], c["m"], c["kind"], c["vw"], rho, nb)
        lam = np.array([orc.fringe_rate(P, x) for x in c["x"][fl, 0]])
        forcing = (c["m"][fl] * lam)[:, None] * (np.array(U) - v[fl]) if fr else 0.0
        rate = (c["m"][fl, None] * (f["a"][fl] - np.array(g))).sum(axis=0) - np.sum(forcing, axis=0)
        scale = np.abs(c["m"][fl, None] * f["a"][fl]).sum()
        np.testing.assert_allclose(F[:2], -rate[:2], rtol=0, atol=1e-12 * scale)
        assert np.abs(F[:2]).max() > 1e-6 * scale            # the walls do take momentum


def test_uniform_flow_drags_the_cylinder_downstream(orc):
    """Uniform flow (U, 0) past the cylinder at rest: the viscous shear at the
    wall pushes the body along +x; by the layout's symmetry about its axis the
    lift is small against the drag."""
    c = _cylinder()
    P = orc.make_params(2, c["lo"], c["L"], c["periodic"], c["rho0"], c["c"], c["eta"], c["h_min"])
    s0 = orc.sigma0_for(c, 2)
    nb = orc.neighbours(P, c["x"], c["h"], "cells")
    rho, _ = orc.density(P, c["x"], c["h"], c["kind"], s0, nb)
    F = orc.wall_force(P, c["x"], c["v"], c["h"], c["m"], c["kind"], c["vw"], rho, nb)
    assert F[0] > 0.0
    assert abs(F[1]) < 0.05 * F[0]
