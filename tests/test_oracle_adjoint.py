"""Pins of the oracle's hand-written adjoint of the step (neighbour lists and
dt frozen) against central finite differences of the oracle's own forward
rollout: directional derivatives of a random linear functional of the final
state (x, v, a, dr) with respect to the initial positions, velocities and the
viscosity, through the initial force pass and several steps.  The cases put
the Riemann dissipation limiter and the transport-velocity limiter in their
active bands, so their subgradients are exercised too."""
import numpy as np
import pytest

from paper_2411_13992_gb300 import cases


def _setup(orc, kind="tgv", tv_mode=1, seed=3):
    if kind == "tgv":
        c = cases.tgv2d(12, jitter_dp=0.12, seed=seed)
    elif kind == "cavity":
        c = cases.cavity2d(10, U=1.0, jitter_dp=0.12, seed=seed)
    else:
        c = cases.tgv3d(7, jitter_dp=0.12, seed=seed)
    P = orc.make_params(c["dim"], c["lo"], c["L"], c["periodic"], c["rho0"], c["c"], c["eta"], c["h_min"],
                        u_ref=c["u_ref"], tv_mode=tv_mode)
    s0 = orc.sigma0_for(c, c["dim"])
    return c, P, s0


def _loss(orc, P, c, s0, dt, x0, v0, T, wts):
    st = orc.rollout(P, c, x0, v0, s0, dt, T, mode="brute")[-1]
    return sum((wts[k] * st[k]).sum() for k in wts)


@pytest.mark.parametrize("kind,tv_mode", [("tgv", 1), ("tgv", 2), ("cavity", 1), ("3d", 1)])
def test_adjoint_matches_central_differences(orc, kind, tv_mode):
    c, P, s0 = _setup(orc, kind, tv_mode)
    rng = np.random.default_rng(7)
    n, D = c["n"], c["dim"]
    fl = (c["kind"] == 0)[:, None].astype(float)
    dt = 0.5 * orc.time_step(P, c["v"], c["kind"])
    T = 3
    wts = {k: np.zeros((n, 3)) for k in ("x", "v", "a", "dr")}
    for k, scale in (("x", 1.0), ("v", 1.0), ("a", 1e-2), ("dr", 1e3)):
        wts[k][:, :D] = rng.standard_normal((n, D)) * scale
    states = orc.rollout(P, c, c["x"], c["v"], s0, dt, T, mode="brute")
    s = P.h_min ** 2 * (states[-1]["R"][:, :D] ** 2).sum(axis=1)
    if tv_mode == 1:
        assert ((s > P.tv_thresh) & (s < 1.0 / P.tv_C)).any()       # limiter band active
    xb, vb, eb = orc.rollout_adjoint(P, c, states, s0, dt, wts, mode="brute")
    dx = np.zeros((n, 3))
    dx[:, :D] = rng.standard_normal((n, D)) * fl
    dv = np.zeros((n, 3))
    dv[:, :D] = rng.standard_normal((n, D)) * fl
    ex = 1e-7 * c["dp"]
    ev = 1e-6
    fd_x = (_loss(orc, P, c, s0, dt, c["x"] + ex * dx, c["v"], T, wts)
            - _loss(orc, P, c, s0, dt, c["x"] - ex * dx, c["v"], T, wts)) / (2 * ex)
    fd_v = (_loss(orc, P, c, s0, dt, c["x"], c["v"] + ev * dv, T, wts)
            - _loss(orc, P, c, s0, dt, c["x"], c["v"] - ev * dv, T, wts)) / (2 * ev)
    eta0 = P.eta
    ee = 1e-3 * eta0                  # eta enters linearly per step: a larger step stays accurate
    P.eta = eta0 + ee
    lp = _loss(orc, P, c, s0, dt, c["x"], c["v"], T, wts)
    P.eta = eta0 - ee
    lm = _loss(orc, P, c, s0, dt, c["x"], c["v"], T, wts)
    P.eta = eta0
    fd_e = (lp - lm) / (2 * ee)
    ad_x, ad_v = (xb * dx).sum(), (vb * dv).sum()
    assert abs(ad_x - fd_x) <= 1e-5 * abs(fd_x), (ad_x, fd_x)
    assert abs(ad_v - fd_v) <= 1e-5 * abs(fd_v), (ad_v, fd_v)
    assert abs(eb - fd_e) <= 1e-5 * abs(fd_e), (eb, fd_e)


def test_second_kernel_derivative(orc):
    for dim in (2, 3):
        h = 0.41
        e = 1e-6 * h
        for q in np.linspace(0.05, 1.95, 20):
            r = q * h
            fd = (orc.kernel_dW(r + e, h, dim) - orc.kernel_dW(r - e, h, dim)) / (2 * e)
            assert abs(fd - orc.kernel_d2W(r, h, dim)) <= 1e-7 * abs(orc.kernel_d2W(0.0, h, dim))


def test_adjoint_cells_and_brute_force_agree(orc):
    c, P, s0 = _setup(orc, "tgv", 1)
    dt = 0.5 * orc.time_step(P, c["v"], c["kind"])
    st = orc.rollout(P, c, c["x"], c["v"], s0, dt, 1)
    cot = {k: np.ones((c["n"], 3)) for k in ("x", "v", "a", "dr")}
    a, ea = orc.step_adjoint(P, c, st[0], s0, dt, cot, mode="cells")
    b, eb = orc.step_adjoint(P, c, st[0], s0, dt, cot, mode="brute")
    for k in a:
        np.testing.assert_allclose(a[k], b[k], rtol=0, atol=1e-12 * np.abs(b[k]).max())
    assert abs(ea - eb) <= 1e-12 * abs(eb)
