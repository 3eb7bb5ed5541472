"""Free-stream forcing and the body force (flow past the cylinder, Sec. 4.4,
Eq. 18) on the GPU against the FP64 oracle, through the C ABI.

The forcing is the fringe-region technique standing in for the free-stream
boundary the paper cites without giving it: lambda(x) (U_inf - v) in a region
of the periodic box (sph_params.fringe_*).  The body force is the force of
the fluid on the wall particles (sph_params.body_force), reported in
sph_diag.body_force; the oracle sums it pair by pair over the fluid's wall
neighbours (oracle.wall_force), the library from the momentum balance of the
fluid's pair terms.  Bounds: FP64 1e-12 per step as in the other parity
tests (1e-9 relative for the body force, a difference of sums); FP32 1e-5
on x, v, rho and 1e-3 on a, dr and the body force."""
import numpy as np
import pytest

import oracle
import paper_2411_13992_gb300 as sph
from paper_2411_13992_gb300 import cases

from gpu_helpers import compare_step, oracle_params, oracle_trajectory

pytestmark = pytest.mark.gpu

U_INF = (1.0, 0.0, 0.0)


def _cylinder():
    # small variable-resolution layout (h ratio 2, walls) with a fringe region downstream
    c = cases.cylinder2d(D=1.0, res=12, box=(6.0, 3.0), center=(2.0, 1.5), refine=(1.0, 4.5, 0.5, 2.5),
                         band_dp=2.0, U=1.0)
    return c, (4.0, (1.0, 0.0, 0.0), (4.6, 5.9, 0.6, 0.4))


def _lib_fringe(fr):
    lam, u, xs = fr
    return {"fringe_lambda": lam, "fringe_u": tuple(u), "fringe_x": tuple(xs)}


def _perturbed(c):
    v = c["v"].copy()
    fl = c["kind"] == 0
    v[fl, 1] += 0.05 * np.sin(2.0 * np.pi * c["x"][fl, 0] / c["L"][0])
    v[fl, 0] -= 0.3 * np.exp(-((c["x"][fl, 0] - 5.2) ** 2))     # a slower stream in the fringe region
    return v


@pytest.mark.parametrize("precision", [64, 32])
def test_step_parity_with_the_fringe_forcing(precision):
    c, fr = _cylinder()
    c = dict(c)
    c["v"] = _perturbed(c)
    dt, states, P, s0 = oracle_trajectory(c, 4, {0, 4}, fringe=fr)
    for k in (0, 4):
        err, ref, _ = compare_step(c, states[k], dt, s0, P, precision=precision, **_lib_fringe(fr))
        if precision == 64:
            for f in ("x", "v", "rho", "ke"):
                assert err[f] <= 1e-12, (k, f, err)
            assert err["a"] <= max(1e-12, 4.0 * err["floor_a"]), err
        else:
            for f in ("x", "v", "rho", "ke"):
                assert err[f] <= 1e-5, (k, f, err)
            assert err["a"] <= 1e-3, err
    # the forcing is not vacuous: it changes the acceleration in the fringe region
    P0 = oracle_params(c)
    ref0 = oracle.step(P0, c, states[4], s0, dt)
    fl = (c["kind"] == 0) & (c["x"][:, 0] > 5.0) & (c["x"][:, 0] < 5.5)
    assert np.abs(ref["a"][fl] - ref0["a"][fl]).max() > 0.1


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("kind", ["cylinder", "cavity"])
def test_body_force_matches_the_oracles_wall_sum(precision, kind):
    if kind == "cylinder":
        c, fr = _cylinder()
        c = dict(c)
        c["v"] = _perturbed(c)
        extra = _lib_fringe(fr)
    else:
        c, fr, extra = cases.cavity2d(32, U=1.0), None, {}
        c = dict(c)
        v = c["v"].copy()
        fl = c["kind"] == 0
        v[fl, 0] = 0.4 * np.sin(np.pi * c["x"][fl, 1]) ** 2
        c["v"] = v
    P = oracle_params(c, fringe=fr)
    s0 = oracle.sigma0_for(c, 2)
    fp = oracle.force_pass(P, c, c["x"], c["v"], s0)
    nb = oracle.neighbours(P, c["x"], c["h"], "cells")
    F = oracle.wall_force(P, c["x"], c["v"], c["h"], c["m"], c["kind"], c["vw"], fp["rho"], nb)
    sim = sph.Simulation(c, precision=precision, body_force=1, **extra)
    try:
        sim.set_state()
        sim.build_cells()                   # the initial force pass on (x, v)
        got = sim.diag()["body_force"]
    finally:
        sim.close()
    tol = 1e-9 if precision == 64 else 1e-3
    assert np.abs(F[:2]).max() > 0.0
    assert np.abs(got[:2] - F[:2]).max() <= tol * np.abs(F[:2]).max(), (got, F)


def test_body_force_is_zero_unless_asked():
    c, fr = _cylinder()
    sim = sph.Simulation(c, precision=32)
    try:
        sim.set_state()
        sim.build_cells()
        assert np.all(sim.diag()["body_force"] == 0.0)
    finally:
        sim.close()


def test_time_and_body_impulse_accumulate_over_the_steps():
    """sph_diag.time is the sum of the steps' dt and body_impulse the sum of
    each step's body force times its dt, both from zero at sph_build_cells."""
    c, fr = _cylinder()
    dt = 2.0e-4
    sim = sph.Simulation(c, precision=64, body_force=1, fixed_dt=dt, graphs=0, **_lib_fringe(fr))
    try:
        sim.set_state()
        sim.build_cells()
        d0 = sim.diag()
        assert d0["time"] == 0.0 and np.all(d0["body_impulse"] == 0.0)
        imp = np.zeros(3)
        for k in range(6):
            sim.step(1)
            d = sim.diag()
            imp += d["body_force"] * dt
            assert d["time"] == pytest.approx((k + 1) * dt, rel=1e-14)
            np.testing.assert_allclose(d["body_impulse"], imp, rtol=1e-13, atol=1e-300)
        assert np.abs(imp[:2]).max() > 0.0
    finally:
        sim.close()
