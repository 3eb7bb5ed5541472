"""Degenerate inputs on the GPU, against the oracle.

* Two distinct particles at exactly the same position (a duplicated
  particle): the pair adds W(0) to sigma and nothing to the forces, the
  residual or the continuity sum (r = 0), in both integrators and both
  precisions.
* Isolated particles (no neighbour within 2h) under gravity: one advection
  step of the dual-criteria integrator lands exactly on x0 + v0 Dt + g Dt^2/2,
  whatever the number of substeps (drift-kick-drift is exact for a constant
  acceleration)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2411_13992_gb300 as sph
from paper_2411_13992_gb300 import cases

from gpu_helpers import compare_step, normwise, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available()


def _with_duplicate(c, k=37):
    for key in ("x", "v", "h", "m", "kind", "vw"):
        c[key] = np.ascontiguousarray(np.concatenate([c[key], c[key][k:k + 1]]))
    c["n"] += 1
    return c


@pytest.mark.parametrize("precision", [64, 32])
def test_coincident_particles_kick_drift_kick(precision):
    c = _with_duplicate(cases.tgv2d(20, jitter_dp=0.05, seed=2))
    P = oracle_params(c)
    s0 = oracle.sigma0_for(c, 2)
    fp = oracle.force_pass(P, c, c["x"], c["v"], s0)
    dt = 0.5 * oracle.time_step(P, c["v"], c["kind"])
    st = {"x": c["x"], "v": c["v"], "a": fp["a"], "dr": fp["dr"]}
    err, ref, got = compare_step(c, st, dt, s0, P, precision=precision)
    print(precision, {k: "%.1e" % v for k, v in err.items() if isinstance(v, float)})
    tol = 1e-12 if precision == 64 else 1e-5
    for k in ("x", "v", "rho"):
        assert err[k] <= tol, (k, err)
    assert np.isfinite(got["a"]).all()


@pytest.mark.parametrize("precision", [64, 32])
def test_coincident_particles_dual_criteria(precision):
    c = _with_duplicate(cases.tgv2d(20, jitter_dp=0.05, seed=2))
    P = oracle_params(c)
    s0 = oracle.sigma0_for(c, 2)
    st = {"x": c["x"], "v": c["v"], "drho": np.zeros(c["n"])}
    ref = oracle.dual_step(P, c, st, s0)
    sim = sph.Simulation(c, precision=precision, integrator=sph.INT_DUAL)
    try:
        sim.set_state()
        sim.build_cells()
        sim.step(1)
        assert sim.sync() is None
        got = sim.get_state()
        d = sim.diag()
    finally:
        sim.close()
    tol = 1e-12 if precision == 64 else 1e-5
    assert d["substeps"] == ref["substeps"]
    assert normwise(got["v"], ref["v"]) <= tol
    assert normwise(got["rho"], ref["rho"]) <= tol


def test_isolated_particles_follow_the_parabola_in_one_advection_step():
    n = 4
    x = np.zeros((n, 3))
    x[:, 0] = 1.0 + 3.9 * np.arange(n)
    x[:, 1] = 5.0
    v = np.zeros((n, 3))
    v[:, 0] = [0.1, -0.2, 0.0, 0.05]
    v[:, 1] = [0.3, 0.0, -0.1, 0.2]
    c = {"name": "isolated", "dim": 2, "n": n, "x": x, "v": v, "h": np.full(n, 1.3), "m": np.ones(n),
         "kind": np.zeros(n, np.int8), "vw": np.zeros((n, 3)), "lo": (0.0, 0.0, 0.0), "L": (20.0, 10.0, 1.0),
         "periodic": (0, 0, 0), "rho0": 1.0, "c": 10.0, "eta": 0.0, "g": (0.0, -0.5, 0.0), "h_min": 1.3,
         "h_max": 1.3, "u_ref": 0.4}
    sim = sph.Simulation(c, precision=64, integrator=sph.INT_DUAL)
    try:
        sim.set_state()
        sim.build_cells()
        sim.step(1)
        assert sim.sync() is None
        got = sim.get_state()
        d = sim.diag()
    finally:
        sim.close()
    Dt = d["dt"]
    assert Dt == pytest.approx(0.25 * 1.3 / 0.4, rel=1e-15)
    g = np.array([0.0, -0.5, 0.0])
    np.testing.assert_allclose(got["x"], x + v * Dt + 0.5 * g * Dt ** 2, rtol=0, atol=1e-13)
    np.testing.assert_allclose(got["v"], v + g * Dt, rtol=0, atol=1e-14)
    assert d["substeps"] >= 2


@pytest.mark.parametrize("precision", [64, 32])
def test_single_particle_falls_freely_with_its_self_density(precision):
    """One particle (the smallest input the library takes): its density is
    its own kernel value, rho0 W(0) / sigma0 with W(0) = 7 / (4 pi h^2) in
    2-D (Wendland C2, Sec. 4); it has no neighbour, so no pressure, viscous
    or correction term, and kick-drift-kick steps of fixed dt under gravity
    land on the parabola x0 + v0 t + g t^2 / 2 (exact for a constant
    acceleration)."""
    h = 1.3
    x = np.array([[4.0, 6.0, 0.0]])
    v = np.array([[0.2, -0.1, 0.0]])
    c = {"name": "single", "dim": 2, "n": 1, "x": x, "v": v, "h": np.full(1, h), "m": np.ones(1),
         "kind": np.zeros(1, np.int8), "vw": np.zeros((1, 3)), "lo": (0.0, 0.0, 0.0), "L": (20.0, 20.0, 1.0),
         "periodic": (0, 0, 0), "rho0": 1.0, "c": 10.0, "eta": 0.01, "g": (0.0, -0.5, 0.0), "h_min": h,
         "h_max": h, "u_ref": 0.4}
    dt, steps = 0.01, 10
    sim = sph.Simulation(c, precision=precision, fixed_dt=dt)
    try:
        sim.set_state()
        sim.build_cells()
        rho0 = sim.get_state()["rho"][0]
        sim.step(steps)
        assert sim.sync() is None
        got = sim.get_state()
    finally:
        sim.close()
    s0 = oracle.sigma0_for(c, 2)[0]
    w0 = 7.0 / (4.0 * np.pi * h * h)
    tol = 1e-14 if precision == 64 else 1e-6
    assert rho0 == pytest.approx(w0 / s0, rel=tol)
    t = steps * dt
    g = np.array([0.0, -0.5, 0.0])
    np.testing.assert_allclose(got["x"], x + v * t + 0.5 * g * t * t, rtol=0, atol=1e-12 if precision == 64 else 1e-6)
    np.testing.assert_allclose(got["v"], v + g * t, rtol=0, atol=1e-13 if precision == 64 else 1e-6)
    assert np.abs(got["dr"]).max() == 0.0
