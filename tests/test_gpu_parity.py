"""GPU parity of libsphtv against the FP64 CPU oracle, through the C ABI.

Contract (per step, from an identical input state, normwise relative
max_i |q_lib - q_orc| / max_i |q_orc| per field):
  FP64 form: x displacement, v, rho and the kinetic energy within 1e-12;
             a and dr within max(1e-12, 4 f), where f is the rounding floor
             of the step on that state: the oracle against itself with every
             neighbour sum reversed (on a near-perfect lattice p = c^2 (rho -
             rho0) is itself rounding noise and f reaches 1e-12); identical
             limiter decisions (chi > 0 set).
  FP32 form: x displacement, v, rho within 1e-5; a and dr within 1e-3.  The
             looser bound on a and dr is the conditioning of the equation of
             state: p = c^2 (rho - rho0) turns the FP32 rounding of the
             cell-relative positions (~6e-8 relative) into a relative error
             of rho - rho0 larger by rho/(rho - rho0) ~ 1e3 on these flows.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2411_13992_gb300 as sph
from paper_2411_13992_gb300 import cases

from gpu_helpers import compare_step, gpu_one_step, normwise, oracle_params, oracle_trajectory

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32_STATE = 1e-5
TOL32_FORCE = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU parity tests need a CUDA device"
    oracle.set_threads(16)
    torch.cuda.set_device(0)


def _assert64(err):
    for k in ("x", "v", "rho", "ke"):
        assert err[k] <= TOL64, (k, err)
    assert err["a"] <= max(TOL64, 4.0 * err["floor_a"]), err
    if err["n_chi_ref"] == 0:
        assert err["dr_abs"] == 0.0, err
    else:
        assert err["dr"] <= max(TOL64, 4.0 * err["floor_dr"]), err
    assert err["n_chi_got"] == err["n_chi_ref"], err
    assert err["near_threshold"] == 0, err


def _assert32(err):
    for k in ("x", "v", "rho"):
        assert err[k] <= TOL32_STATE, (k, err)
    assert err["a"] <= TOL32_FORCE, err
    if err["n_chi_ref"]:
        assert err["dr"] <= TOL32_FORCE, err
    assert err["ke"] <= TOL32_STATE, err


# ------------------------------------------------------------ 2-D Taylor-Green

@pytest.fixture(scope="module")
def tgv2d_traj():
    c = cases.tgv2d(50)
    dt, states, P, s0 = oracle_trajectory(c, 100, {0, 1, 20, 60, 100})
    return c, dt, states, P, s0


@pytest.mark.parametrize("k", [0, 1, 20, 60, 100])
def test_fp64_step_parity_tgv2d(tgv2d_traj, k):
    c, dt, states, P, s0 = tgv2d_traj
    err, _, _ = compare_step(c, states[k], dt, s0, P, precision=64)
    _assert64(err)


@pytest.mark.parametrize("mode", [oracle.TV_UNLIMITED, oracle.TV_BACKGROUND, oracle.TV_NONE])
def test_fp64_step_parity_other_correction_modes(tgv2d_traj, mode):
    c, dt, states, P0, s0 = tgv2d_traj
    P = oracle_params(c, tv_mode=mode)
    for k in (20, 100):
        err, _, _ = compare_step(c, states[k], dt, s0, P, precision=64, tv_mode=mode)
        _assert64(err)
        err, _, _ = compare_step(c, states[k], dt, s0, P, precision=32, tv_mode=mode)
        _assert32(err)


@pytest.mark.parametrize("k", [0, 20, 100])
def test_fp32_step_parity_tgv2d(tgv2d_traj, k):
    c, dt, states, P, s0 = tgv2d_traj
    err, _, _ = compare_step(c, states[k], dt, s0, P, precision=32)
    _assert32(err)


def test_limiter_is_active_in_the_parity_states(tgv2d_traj):
    c, dt, states, P, s0 = tgv2d_traj
    err, _, _ = compare_step(c, states[100], dt, s0, P, precision=64)
    assert err["n_chi_ref"] > 0


def test_initial_force_pass_and_first_dt(tgv2d_traj):
    c, dt, states, P, s0 = tgv2d_traj
    sim = sph.Simulation(c, precision=64)
    sim.set_state()
    sim.build_cells()
    sim.sync()
    g, d = sim.get_state(), sim.diag()
    sim.close()
    ref = states[0]
    start, idx = oracle.neighbours(P, c["x"], c["h"])
    alt = oracle.forces(P, c["x"], c["v"], c["h"], c["m"], c["kind"], c["vw"], ref["rho"],
                        (start, oracle.reverse_segments(start, idx)))
    floor_a = normwise(alt["a"], ref["a"])
    assert normwise(g["a"], ref["a"]) <= max(TOL64, 4.0 * floor_a)
    assert normwise(g["rho"], ref["rho"]) <= TOL64
    assert np.array_equal(g["x"], c["x"])               # no drift in the initial pass
    assert abs(d["dt_next"] - dt) <= 1e-14 * dt


# --------------------------------------------------------- 3-D, walls, ragged

@pytest.mark.parametrize("n", [16, 15])
def test_step_parity_tgv3d(n):
    c = cases.tgv3d(n)
    dt, states, P, s0 = oracle_trajectory(c, 5, {0, 5})
    for k in (0, 5):
        err, _, _ = compare_step(c, states[k], dt, s0, P, precision=64)
        _assert64(err)
        err, _, _ = compare_step(c, states[k], dt, s0, P, precision=32)
        _assert32(err)


def test_step_parity_cavity_walls_and_gravity():
    c = cases.cavity2d(32, U=1.0)
    c["g"] = (0.0, -0.5, 0.0)
    dt, states, P, s0 = oracle_trajectory(c, 20, {0, 20})
    for k in (0, 20):
        err, _, _ = compare_step(c, states[k], dt, s0, P, precision=64)
        _assert64(err)
    assert err["n_chi_ref"] > 0                          # walls disorder the fluid: limiter active


def test_step_parity_cavity_low_velocity_lid():
    c = cases.cavity2d(24, U=1.0e-3)
    dt, states, P, s0 = oracle_trajectory(c, 10, {10})
    err, _, _ = compare_step(c, states[10], dt, s0, P, precision=64)
    _assert64(err)


def _small_cylinder():
    return cases.cylinder2d(D=1.0, res=12, box=(4.0, 2.5), center=(1.5, 1.25), refine=(1.0, 3.5, 0.5, 2.0),
                            band_dp=2.0)


@pytest.mark.parametrize("opts", [{}, {"tv_h_per_particle": True}, {"h_pair_max": True},
                                  {"tv_mode": oracle.TV_UNLIMITED}, {"tv_mode": oracle.TV_BACKGROUND}])
def test_step_parity_variable_resolution(opts):
    c = _small_cylinder()
    assert c["h_max"] > 1.5 * c["h_min"]
    dt, states, P, s0 = oracle_trajectory(c, 8, {0, 8}, **opts)
    for k in (0, 8):
        err, _, _ = compare_step(c, states[k], dt, s0, P, precision=64, **opts)
        _assert64(err)
        err, _, _ = compare_step(c, states[k], dt, s0, P, precision=32, **opts)
        _assert32(err)


# --------------------------------------------------------------- edge cases

def test_single_particle():
    c = cases.lattice_block(2, 1, dp=0.1)
    c["L"] = (1.0, 1.0, 1.0)
    c["g"] = (0.0, -1.0, 0.0)
    c["h_min"] = c["h_max"] = 0.13
    P = oracle_params(c)
    s0 = oracle.sigma0_for(c, 2)
    fp = oracle.force_pass(P, c, c["x"], c["v"], s0)
    dt = 1.0e-3
    st = {"x": c["x"], "v": c["v"], "a": fp["a"], "dr": fp["dr"]}
    ref = oracle.step(P, c, st, s0, dt)
    got, _ = gpu_one_step(c, st, dt, 64)
    np.testing.assert_allclose(got["v"], ref["v"], rtol=1e-15, atol=0)
    np.testing.assert_allclose(got["rho"], ref["rho"], rtol=1e-14)
    assert got["a"][0, 1] == -1.0


def test_particles_on_cell_and_periodic_boundaries():
    """A perfect lattice whose rows sit on x = 0 and on cell edges: 39 rows
    at k dp with 15 cells of edge 1/15, so rows k = 13 and 26 lie on the
    edges x = 1/3 and 2/3."""
    c = cases.tgv2d(39, jitter_dp=0.0)
    c["x"][:, :2] -= 0.5 * c["dp"]                        # rows at k dp: x = 0 and cell edges exactly
    c["x"][:, :2] = np.mod(c["x"][:, :2], 1.0)
    dt, states, P, s0 = oracle_trajectory(c, 3, {0, 3})
    for k in (0, 3):
        err, _, _ = compare_step(c, states[k], dt, s0, P, precision=64)
        _assert64(err)


def test_sparse_layout_with_empty_cells():
    c = cases.tgv2d(40)
    keep = (c["x"][:, 0] < 0.45) | (c["x"][:, 1] > 0.8)
    for key in ("x", "v", "h", "m", "kind", "vw"):
        c[key] = np.ascontiguousarray(c[key][keep])
    c["n"] = int(keep.sum())
    dt, states, P, s0 = oracle_trajectory(c, 4, {4})
    err, _, _ = compare_step(c, states[4], dt, s0, P, precision=64)
    _assert64(err)


def test_deterministic_and_order_independent():
    c = cases.tgv2d(40)
    runs = []
    for perm in (None, None, np.random.default_rng(1).permutation(c["n"])):
        cc = dict(c)
        if perm is not None:
            for key in ("x", "v", "h", "m", "kind", "vw"):
                cc[key] = np.ascontiguousarray(c[key][perm])
        sim = sph.Simulation(cc, precision=32)
        sim.set_state()
        sim.build_cells()
        sim.step(10)
        sim.sync()
        g = sim.get_state()
        sim.close()
        if perm is not None:
            inv = np.argsort(perm)
            g = {k: v[inv] for k, v in g.items()}
        runs.append(g)
    for k in ("x", "v", "a", "rho"):
        assert np.array_equal(runs[0][k], runs[1][k]), k           # bitwise rerun
        tol = TOL32_FORCE if k == "a" else TOL32_STATE            # input order changes sums only
        assert normwise(runs[2][k], runs[0][k]) <= tol, k


def test_state_round_trip_is_exact():
    c = cases.tgv3d(12)
    for prec in (64, 32):
        sim = sph.Simulation(c, precision=prec)
        sim.set_state()
        sim.build_cells()
        sim.sync()
        g = sim.get_state()
        sim.close()
        assert np.array_equal(g["x"], c["x"])
        if prec == 64:
            assert np.array_equal(g["v"], c["v"])


# ------------------------------------------------------- errors, not faults

def test_device_errors_are_reported_not_trapped():
    c = cases.tgv2d(20)
    v = c["v"].copy()
    v[7, 0] = np.nan
    sim = sph.Simulation(c, precision=64, fixed_dt=1e-3)
    sim.set_state(v=v)
    sim.build_cells()
    sim.step(1)
    with pytest.raises(sph.SphError) as e:
        sim.sync()
    assert e.value.status == 5                              # SPH_ERR_NAN
    sim.sync()                                              # the error word was cleared
    sim.close()
    cv = cases.cavity2d(16)
    x = cv["x"].copy()
    x[3, 1] = 5.0                                           # outside the non-periodic box
    sim = sph.Simulation(cv, precision=32)
    sim.set_state(x=x)
    sim.build_cells()
    with pytest.raises(sph.SphError) as e:
        sim.sync()
    assert e.value.status == 6                              # SPH_ERR_DOMAIN
    sim.close()
    torch.cuda.synchronize()                                # the context is still usable


def test_call_order_and_argument_errors():
    c = cases.tgv2d(20)
    sim = sph.Simulation(c, precision=64)
    with pytest.raises(sph.SphError) as e:
        sim.step(1)
    assert e.value.status == 7                              # SPH_ERR_STATE
    with pytest.raises(sph.SphError) as e:
        sph.sph_set_state(sim.ctx, c["x"], c["v"], c["v"], None, c["h"], c["m"])
    assert e.value.status == 1
    with pytest.raises(sph.SphError):
        sim.set_dt(-1.0)
    sim.close()


# ------------------------------------------------- multi-step and decay rate

def _ke_series(c, nsteps, precision, dt):
    sim = sph.Simulation(c, precision=precision, fixed_dt=dt)
    sim.set_state()
    sim.build_cells()
    ke = [sim.diag()["ke"]]
    for _ in range(nsteps):
        sim.step(1)
        ke.append(sim.diag()["ke"])
    sim.sync()
    g = sim.get_state()
    sim.close()
    return np.array(ke), g


def test_multistep_trajectory_and_decay_rates(tgv2d_traj):
    c, dt, states, P, s0 = tgv2d_traj
    ke64, g64 = _ke_series(c, 100, 64, dt)
    ke32, g32 = _ke_series(c, 100, 32, dt)
    ref = states[100]
    # 100 steps of chaotic particle dynamics: rounding differences grow, stay small
    assert normwise(g64["v"], ref["v"]) < 1e-9
    assert normwise(g32["v"], ref["v"]) < 1e-3
    t = dt * np.arange(101)
    rate64 = np.polyfit(t, np.log(ke64), 1)[0]
    rate32 = np.polyfit(t, np.log(ke32), 1)[0]
    orc_ke = []
    st = {"x": c["x"], "v": c["v"], "a": states[0]["a"], "dr": states[0]["dr"]}
    for _ in range(100):
        orc_ke.append(0.5 * (c["m"][:, None] * st["v"] ** 2).sum())
        st = oracle.step(P, c, st, s0, dt)
    orc_ke.append(0.5 * (c["m"][:, None] * st["v"] ** 2).sum())
    rate_orc = np.polyfit(t, np.log(np.array(orc_ke)), 1)[0]
    assert abs(rate64 / rate_orc - 1.0) < 1e-9
    assert abs(rate32 / rate64 - 1.0) < 1e-3               # FP32 decay rate within 1e-3 of FP64
    assert rate64 < 0 and math.isfinite(rate32)


def _build_and_step(c, precision, ad, rho_first):
    sim = sph.Simulation(c, precision=precision)
    try:
        if ad is None:
            sim.set_state()
        else:
            sim.set_state(a=ad["a"], dr=ad["dr"])
        sim.build_cells()
        first = sim.get_state() if rho_first else None
        d0 = sim.diag()
        sim.step(3)
        assert sim.sync() is None
        return first, d0, sim.get_state(), sim.diag()
    finally:
        sim.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_build_with_a_and_dr_given_leaves_the_sort_to_the_first_step(precision):
    """With a and dr given, sph_build_cells computes only the diagnostics
    and dt_0; the first step sorts the particles itself.  The densities
    reported before any step (sorted on demand) and the states after three
    steps are bit for bit those of a build that computed a and dr itself,
    whether or not the densities were asked for first."""
    c = cases.tgv2d(40, jitter_dp=0.05, seed=6)
    full_first, full_d0, full_after, full_d = _build_and_step(c, precision, None, True)
    ad = {"a": full_first["a"], "dr": full_first["dr"]}
    lazy_first, lazy_d0, lazy_after, lazy_d = _build_and_step(c, precision, ad, True)
    _, _, direct_after, _ = _build_and_step(c, precision, ad, False)
    assert np.array_equal(lazy_first["rho"], full_first["rho"])
    assert lazy_d0["dt_next"] == full_d0["dt_next"] and lazy_d0["vmax"] == full_d0["vmax"]
    for k in ("x", "v", "a", "dr", "rho"):
        assert np.array_equal(lazy_after[k], full_after[k]), k
        assert np.array_equal(direct_after[k], full_after[k]), k
    assert lazy_d["steps"] == full_d["steps"] == 3
