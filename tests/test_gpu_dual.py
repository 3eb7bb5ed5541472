"""GPU parity of the dual-criteria integrator (Sec. 2.4, SPH_INT_DUAL) with
the oracle's dual step.

One advection step from the same state (x, v and the carried d rho/dt) on
both sides: the substep count and Dt_ad must agree exactly, x displacement,
v and rho normwise within the FP64 tolerance of the kick-drift-kick parity
(1e-12), the density rate, acceleration and correction within 1e-11
(the equation of state divides by rho - rho0; measured <= 2.5e-13).  The FP32 form is held to 1e-5 on x, v, rho like the
kick-drift-kick FP32 form.  Also: several advection steps in a row, the
density-rate round trip through the ABI, and momentum conservation of the
full-size FP32 step."""
import numpy as np
import pytest
import torch

import oracle
import paper_2411_13992_gb300 as sph
from paper_2411_13992_gb300 import cases

from gpu_helpers import lib_overrides, normwise, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available()
    oracle.set_threads(16)


def _case(kind):
    if kind == "tgv":
        return cases.tgv2d(24, jitter_dp=0.1, seed=3)
    if kind == "cavity":
        return cases.cavity2d(24, U=1.0, jitter_dp=0.1, seed=3)
    if kind == "cavity_g":
        c = cases.cavity2d(24, U=1.0, jitter_dp=0.1, seed=4)
        c["g"] = (0.0, -1.0, 0.0)
        return c
    if kind == "3d":
        return cases.tgv3d(10, jitter_dp=0.1, seed=3)
    return cases.cylinder2d(D=1.0, res=10, box=(3.0, 2.0), center=(1.0, 1.0), refine=(0.6, 2.4, 0.4, 1.6),
                            band_dp=2.0, jitter_dp=0.05)


def _disp(c, x1, x0):
    d = x1 - x0
    L = np.array(c["L"])
    for k in range(c["dim"]):
        if c["periodic"][k]:
            d[:, k] -= L[k] * np.round(d[:, k] / L[k])
    return d


def _gpu_dual(c, state, precision, steps=1, **kw):
    sim = sph.Simulation(c, precision=precision, integrator=sph.INT_DUAL, **lib_overrides(**kw))
    try:
        sim.set_state(x=state["x"], v=state["v"], drho=state["drho"])
        sim.build_cells()
        sim.step(steps)
        assert sim.sync() is None
        g = sim.get_state()
        g["drho"] = sim.density_rate()
        return g, sim.diag()
    finally:
        sim.close()


def _start_state(c, P, s0, warm=1):
    """A state with a nonzero carried density rate: the oracle's dual step
    from the case's initial state."""
    st = {"x": c["x"], "v": c["v"], "drho": np.zeros(c["n"])}
    for _ in range(warm):
        st = oracle.dual_step(P, c, st, s0)
    return st


def _errors(c, st, ref, got):
    fl = c["kind"] == 0
    return {
        "x": normwise(_disp(c, got["x"], st["x"])[fl], _disp(c, ref["x"], st["x"])[fl]),
        "v": normwise(got["v"][fl], ref["v"][fl]),
        "rho": normwise(got["rho"][fl], ref["rho"][fl]),
        "rho_dev": normwise(got["rho"][fl] - c["rho0"], ref["rho"][fl] - c["rho0"]),
        "drho": normwise(got["drho"][fl], ref["drho"][fl]),
        "a": normwise(got["a"][fl], ref["a"][fl]),
        "dr": normwise(got["dr"][fl], ref["dr"][fl]) if np.abs(ref["dr"][fl]).max() > 0
        else float(np.abs(got["dr"][fl]).max()),
    }


MODES = {"limited": {}, "unlimited": {"tv_mode": oracle.TV_UNLIMITED},
         "background": {"tv_mode": oracle.TV_BACKGROUND}, "none": {"tv_mode": oracle.TV_NONE}}


@pytest.mark.parametrize("kind", ["tgv", "cavity", "cavity_g", "3d", "cylinder"])
@pytest.mark.parametrize("mode", list(MODES))
def test_fp64_advection_step_parity(kind, mode):
    if kind in ("3d", "cylinder", "cavity_g") and mode in ("none", "background"):
        pytest.skip("covered on the 2-D cases")
    c = _case(kind)
    P = oracle_params(c, **MODES[mode])
    s0 = oracle.sigma0_for(c, c["dim"])
    st = _start_state(c, P, s0)
    ref = oracle.dual_step(P, c, st, s0)
    got, diag = _gpu_dual(c, st, 64, **MODES[mode])
    err = _errors(c, st, ref, got)
    print(kind, mode, "substeps", ref["substeps"], diag["substeps"], {k: "%.1e" % v for k, v in err.items()})
    assert diag["substeps"] == ref["substeps"]
    assert diag["dt"] == pytest.approx(ref["Dt"], rel=1e-14)
    for k in ("x", "v", "rho"):
        assert err[k] <= 1e-12, (k, err)
    # rho - rho0, d rho/dt and the pressure force carry the EOS conditioning:
    # rho - rho0 is 1e-2 .. 1e-3 of rho, so their relative rounding is up to
    # 1e3 times that of rho (measured <= 2.5e-13)
    for k in ("rho_dev", "drho", "a", "dr"):
        assert err[k] <= 1e-11, (k, err)


@pytest.mark.parametrize("kind", ["tgv", "cavity", "cavity_g", "3d", "cylinder"])
def test_fp32_advection_step_parity(kind):
    c = _case(kind)
    P = oracle_params(c)
    s0 = oracle.sigma0_for(c, c["dim"])
    st = _start_state(c, P, s0)
    ref = oracle.dual_step(P, c, st, s0)
    got, diag = _gpu_dual(c, st, 32)
    err = _errors(c, st, ref, got)
    print(kind, "FP32 substeps", ref["substeps"], diag["substeps"], {k: "%.1e" % v for k, v in err.items()})
    assert diag["substeps"] == ref["substeps"]
    for k in ("x", "v", "rho"):
        assert err[k] <= 1e-5, (k, err)
    # the same EOS conditioning as the kick-drift-kick FP32 form (1e-3;
    # measured <= 1e-5 here, where rho - rho0 is larger)
    for k in ("drho", "a"):
        assert err[k] <= 1e-3, (k, err)


def test_fp64_several_advection_steps():
    c = _case("tgv")
    P = oracle_params(c)
    s0 = oracle.sigma0_for(c, 2)
    st0 = {"x": c["x"], "v": c["v"], "drho": np.zeros(c["n"])}
    ref = st0
    subs = 0
    for _ in range(6):
        ref = oracle.dual_step(P, c, ref, s0)
        subs += ref["substeps"]
    got, diag = _gpu_dual(c, st0, 64, steps=6)
    err = _errors(c, st0, ref, got)
    print("6 advection steps", subs, {k: "%.1e" % v for k, v in err.items()})
    assert diag["steps"] == 6
    for k in ("x", "v", "rho"):
        assert err[k] <= 1e-10, (k, err)


def test_density_rate_round_trip_and_zero_default():
    c = _case("cavity")
    sim = sph.Simulation(c, precision=64, integrator=sph.INT_DUAL)
    try:
        sim.set_state()
        assert np.abs(sim.density_rate()).max() == 0.0
        sim.close()
        sim = sph.Simulation(c, precision=64, integrator=sph.INT_DUAL)
        rng = np.random.default_rng(1)
        d = rng.standard_normal(c["n"])
        sim.set_state(drho=d)
        sim.build_cells()
        back = sim.density_rate()
        fl = c["kind"] == 0
        np.testing.assert_array_equal(back[fl], d[fl])
        assert np.abs(back[~fl]).max() == 0.0
        with pytest.raises(sph.SphError):
            sph.sph_set_density_rate(sim.ctx, d)          # after build_cells: SPH_ERR_STATE
    finally:
        sim.close()


def test_full_size_fp32_dual_step_conserves_momentum():
    c = cases.tgv3d(64)
    sim = sph.Simulation(c, precision=32, integrator=sph.INT_DUAL)
    try:
        sim.set_state()
        sim.build_cells()
        d0 = sim.diag()
        sim.step(3)
        assert sim.sync() is None
        d1 = sim.diag()
    finally:
        sim.close()
    print("3-D TGV 64^3 dual: substeps per advection step", d1["substeps"], "Dt", d1["dt"])
    assert d1["steps"] == 3 and d1["substeps"] >= 4
    assert d1["mass"] == pytest.approx(d0["mass"], rel=1e-14)     # sums in another block order
    assert np.abs(d1["momentum"] - d0["momentum"]).max() < 1e-5 * d0["mass"] * d0["vmax"]
    assert 0.0 < d1["ke"] < d0["ke"]
