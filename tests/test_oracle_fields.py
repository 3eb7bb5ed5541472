"""Pins of the oracle's density, force and residual sums against fields whose
continuum answer is known: a perfect lattice (Eq. 8 gives rho0 exactly, the
residual of Eq. 14 vanishes), a linear pressure field (Eq. 3 must give
-grad p / rho), a quadratic velocity field (Eq. 7 must give nu lap v) and a
linear density (the residual must give grad(rho0/rho)).  A wrong factor of 2
or a wrong sign in Eq. 3, Eq. 7 or Eq. 14 moves these by 100 %; the lattice
discretisation moves them by under 3 %."""
import numpy as np
import pytest

from paper_2411_13992_gb300 import cases


def _lattice(orc, dim, n, periodic=True, eta=0.0, c0=10.0):
    c = cases.lattice_block(dim, n, dp=1.0, periodic=periodic)
    P = orc.make_params(dim, c["lo"], c["L"], c["periodic"], 1.0, c0, eta, c["h_min"], tv_mode=2)
    return c, P


def _interior(c, dim, margin):
    x = c["x"]
    L = c["L"]
    ok = np.ones(len(x), bool)
    for d in range(dim):
        ok &= (x[:, d] > margin) & (x[:, d] < L[d] - margin)
    return ok


@pytest.mark.parametrize("dim,n", [(2, 12), (3, 8)])
def test_perfect_lattice_is_a_fixed_point(orc, dim, n):
    c, P = _lattice(orc, dim, n)
    s0 = orc.sigma0_for(c, dim)
    out = orc.force_pass(P, c, c["x"], c["v"], s0, mode="brute")
    np.testing.assert_allclose(out["rho"], 1.0, rtol=0, atol=1e-14)
    assert np.abs(out["R"]).max() < 1e-13          # residual scale ~ 1/h ~ 1
    assert np.abs(out["dr"]).max() < 1e-13
    assert np.abs(out["a"]).max() < 1e-11          # rho = rho0 -> p = 0 up to rounding


@pytest.mark.parametrize("dim,n", [(2, 30), (3, 14)])
def test_linear_pressure_gives_minus_grad_p_over_rho(orc, dim, n):
    c, P = _lattice(orc, dim, n, periodic=False)
    x = c["x"]
    G = 1.0e-3
    rho = 1.0 + G * x[:, 0] / 100.0                 # p = c^2 (rho - 1) = G x
    nb = orc.neighbours(P, x, c["h"], "brute")
    f = orc.forces(P, x, np.zeros_like(x), c["h"], c["m"], c["kind"], c["vw"], rho, nb)
    inner = _interior(c, dim, 3.5)
    ratio = f["a"][inner, 0] * rho[inner] / (-G)
    assert 0.97 < ratio.mean() < 1.0, ratio.mean()
    assert ratio.std() < 1e-3
    assert np.abs(f["a"][inner, 1:dim]).max() < 1e-9


@pytest.mark.parametrize("dim,n", [(2, 30), (3, 14)])
def test_quadratic_velocity_gives_nu_laplacian(orc, dim, n):
    eta = 0.5
    c, P = _lattice(orc, dim, n, periodic=False, eta=eta)
    P.riemann_eta = 0.0                              # isolate Eq. 7 from the O(dU^2) Riemann term
    x = c["x"]
    eps = 1.0e-4
    y0 = 0.5 * c["L"][1]
    v = np.zeros_like(x)
    v[:, 0] = eps * (x[:, 1] - y0) ** 2              # lap u = 2 eps
    nb = orc.neighbours(P, x, c["h"], "brute")
    f = orc.forces(P, x, v, c["h"], c["m"], c["kind"], c["vw"], np.ones(len(x)), nb)
    inner = _interior(c, dim, 3.5)
    ratio = f["a"][inner, 0] / (eta * 2.0 * eps)
    assert 0.96 < ratio.mean() < 1.0, ratio.mean()
    assert np.abs(f["a"][inner, 1]).max() < 1e-3 * eta * 2 * eps


@pytest.mark.parametrize("dim,n", [(2, 30), (3, 14)])
def test_residual_of_linear_density_is_grad_of_inverse_density(orc, dim, n):
    """R_i = sum_j (m_j/rho_j) grad_i W_ij on a uniform lattice approximates
    grad(rho0/rho): it points to where particles carry more volume."""
    c, P = _lattice(orc, dim, n, periodic=False)
    x = c["x"]
    G = 1.0e-3
    rho = 1.0 / (1.0 + G * x[:, 0])                  # rho0/rho = 1 + G x
    nb = orc.neighbours(P, x, c["h"], "brute")
    f = orc.forces(P, x, np.zeros_like(x), c["h"], c["m"], c["kind"], c["vw"], rho, nb)
    inner = _interior(c, dim, 3.5)
    ratio = f["R"][inner, 0] / G
    assert 0.97 < ratio.mean() < 1.0, ratio.mean()


def _displaced(orc, dim, n, hdp, delta=1e-4, **kw):
    c = cases.lattice_block(dim, n, dp=1.0, h_over_dp=hdp)
    P = orc.make_params(dim, c["lo"], c["L"], c["periodic"], 1.0, 10.0, 0.0, c["h_min"], tv_mode=2)
    for k, v in kw.items():
        setattr(P, k, v)
    x = c["x"].copy()
    k = len(x) // 2 + n // 2
    x[k, 0] += delta
    out = orc.force_pass(P, c, x, c["v"], orc.sigma0_for(c, dim), mode="cells")
    return out, k, c


@pytest.mark.parametrize("dim,n", [(2, 10), (3, 8)])
def test_transport_correction_restores_a_displaced_particle(orc, dim, n):
    """Displace one lattice particle by delta: the correction of Eq. 14 moves
    it back by a fraction of delta, without overshooting the lattice site.
    A sign error in R or xi pushes it further away."""
    delta = 1e-4
    out, k, _ = _displaced(orc, dim, n, 1.3, delta)
    frac = -out["dr"][k, 0] / delta
    assert 0.02 < frac < 1.0, frac
    assert abs(out["dr"][k, 1]) < 1e-6 * abs(out["dr"][k, 0])


def test_transport_correction_scales_with_xi_and_h_min_squared(orc):
    """Eq. 14/16: dr = xi chi h_min^2 R; R does not depend on h_min or xi."""
    base, k, _ = _displaced(orc, 2, 10, 1.3)
    dbl_h, _, _ = _displaced(orc, 2, 10, 1.3, h_min=2.0 * 1.3)
    dbl_xi, _, _ = _displaced(orc, 2, 10, 1.3, tv_xi=-0.4)
    np.testing.assert_allclose(dbl_h["dr"][k], 4.0 * base["dr"][k], rtol=1e-12)
    np.testing.assert_allclose(dbl_xi["dr"][k], 2.0 * base["dr"][k], rtol=1e-12)
    # limited (Eq. 15-16): this small disorder is below the threshold -> no correction
    lim, _, _ = _displaced(orc, 2, 10, 1.3, tv_mode=1)
    assert np.abs(lim["dr"]).max() == 0.0 and np.abs(lim["R"][k]).max() > 0


def test_restoring_coefficient_approaches_its_continuum_linearisation(orc):
    """Linearising R_k in the displacement delta of particle k gives two
    terms: the kernel Hessian summed over the other particles, which tends to
    -V W''(0) I (the full lattice sum of the Hessian tends to its integral,
    zero), and the change of the neighbours' volumes m/rho_j through their
    densities, which tends to -(V / (S D)) int |grad W|^2 I.  The Wendland C2
    kernel has an r^3 term at the origin, so the Hessian sum converges only
    algebraically in h/dp: the measured coefficient must approach the
    linearisation as h/dp grows (2-D)."""
    import math
    from scipy.integrate import quad
    ratios = []
    for n, hdp in ((20, 3.0), (40, 6.0)):
        delta = 1e-4
        out, k, c = _displaced(orc, 2, n, hdp, delta)
        h = c["h_min"]
        e = 1e-5 * h
        w2 = (orc.kernel_dW(e, h, 2) - orc.kernel_dW(0.0, h, 2)) / e
        integ = quad(lambda r: orc.kernel_dW(r, h, 2) ** 2 * 2 * math.pi * r, 0, 2 * h, epsrel=1e-12)[0]
        K = -w2 - integ / (orc.lattice_sum(2, hdp) * 2)
        ratios.append((-out["dr"][k, 0] / delta) / (0.2 * h * h * K))
    assert 0.75 < ratios[0] < ratios[1] < 1.0, ratios
    assert ratios[1] > 0.9, ratios
