"""Pins of the oracle's Wendland C2 kernel (Sec. 4, h = 1.3 dp) and of the
perfect-lattice reference sum of Eq. 8.  Each check uses a fact that does not
come from the oracle's own formulas: normalisation by adaptive quadrature,
the derivative by finite differences, and the convergence of a lattice sum
to the integral."""
import math

import numpy as np
import pytest
from scipy.integrate import quad


def _shell(dim):
    return (lambda r: 2.0 * math.pi * r) if dim == 2 else (lambda r: 4.0 * math.pi * r * r)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("h", [0.013, 0.7, 2.5])
def test_kernel_integrates_to_one(orc, dim, h):
    shell = _shell(dim)
    val, _ = quad(lambda r: orc.kernel_W(r, h, dim) * shell(r), 0.0, 2.0 * h, epsabs=0.0, epsrel=1e-13,
                  limit=200)
    assert abs(val - 1.0) < 1e-11


@pytest.mark.parametrize("dim", [2, 3])
def test_kernel_derivative_matches_central_difference(orc, dim):
    h = 0.37
    eps = 1e-6 * h
    for q in np.linspace(0.01, 1.99, 41):
        r = q * h
        fd = (orc.kernel_W(r + eps, h, dim) - orc.kernel_W(r - eps, h, dim)) / (2 * eps)
        an = orc.kernel_dW(r, h, dim)
        assert abs(fd - an) <= 1e-7 * abs(orc.kernel_dW(0.5 * h, h, dim)), (q, fd, an)


@pytest.mark.parametrize("dim", [2, 3])
def test_kernel_support_monotone_and_smooth(orc, dim):
    h = 1.1
    assert orc.kernel_W(2.0 * h, h, dim) == 0.0
    assert orc.kernel_dW(2.0 * h, h, dim) == 0.0
    assert orc.kernel_W(2.3 * h, h, dim) == 0.0
    assert orc.kernel_dW(0.0, h, dim) == 0.0
    qs = np.linspace(0.0, 2.0, 201)
    w = np.array([orc.kernel_W(q * h, h, dim) for q in qs])
    dw = np.array([orc.kernel_dW(q * h, h, dim) for q in qs])
    assert np.all(np.diff(w) < 0.0)
    assert np.all(dw <= 0.0)
    # C2 at the edge of the support: W'' -> 0 as q -> 2 (second difference of dW)
    e = 1e-4 * h
    d2 = (orc.kernel_dW(2.0 * h - e, h, dim) - orc.kernel_dW(2.0 * h - 2 * e, h, dim)) / e
    assert abs(d2) < 1e-6 * abs(orc.kernel_dW(0.5 * h, h, dim)) / h


@pytest.mark.parametrize("dim", [2, 3])
def test_lattice_sum_converges_to_the_integral(orc, dim):
    """sum_k W(|k| dp) dp^D -> int W = 1 as h/dp grows; the error of a lattice
    sum of a C2 Wendland function falls like (h/dp)^-(D+3)."""
    errs = [abs(orc.lattice_sum(dim, r) - 1.0) for r in (2.0, 4.0, 8.0)]
    assert errs[1] < 1e-4
    assert errs[2] < errs[1] / 16.0
    assert errs[1] < errs[0] / 16.0
    s13 = orc.lattice_sum(dim, 1.3)
    assert 1.0 < s13 < 1.02      # h = 1.3 dp: within 2 % of the integral


def test_lattice_sum_is_the_density_of_a_perfect_lattice(orc):
    """On a periodic lattice, sum_j V_j W_ij (self included) equals the
    lattice sum for every particle: the two are computed by different oracle
    paths (lattice loop vs neighbour search + density)."""
    from paper_2411_13992_gb300 import cases
    for dim, n in ((2, 12), (3, 8)):
        c = cases.lattice_block(dim, n, dp=0.5)
        P = orc.make_params(dim, c["lo"], c["L"], c["periodic"], 1.0, 10.0, 0.0, c["h_min"])
        nb = orc.neighbours(P, c["x"], c["h"], "brute")
        _, sigma = orc.density(P, c["x"], c["h"], c["kind"], np.ones(c["n"]), nb)
        np.testing.assert_allclose(sigma * c["dp"] ** dim, orc.lattice_sum(dim, 1.3), rtol=1e-13)


@pytest.mark.parametrize("dim,expected,count", [(2, 1.010473, 21), (3, 1.009501, 81)])
def test_lattice_sum_at_h_1p3_by_direct_summation(orc, dim, expected, count):
    """sigma0 dp^D at h = 1.3 dp (Sec. 4) on the unit square / cubic lattice,
    self included: a direct loop over the integer vectors k with |k| < 2.6
    (21 in 2-D, 81 in 3-D) in 40-digit arithmetic with the Wendland C2 form
    W = a_D h^-D (1 - q/2)^4 (2q + 1), whose normalisation a_D is pinned by
    quadrature above.  A wrong shell, a dropped self term or a wrong support
    fails it; the 6-digit values are the ones computed independently before
    the oracle was written."""
    import itertools
    import mpmath
    mpmath.mp.dps = 40
    h = mpmath.mpf("1.3")
    a = mpmath.mpf(7) / (4 * mpmath.pi) if dim == 2 else mpmath.mpf(21) / (16 * mpmath.pi)
    total, terms = mpmath.mpf(0), 0
    for k in itertools.product(range(-3, 4), repeat=dim):
        r = mpmath.sqrt(sum(mpmath.mpf(t) ** 2 for t in k))
        q = r / h
        if q < 2:
            total += a / h ** dim * (1 - q / 2) ** 4 * (2 * q + 1)
            terms += 1
    assert terms == count
    assert abs(float(total) - expected) < 5e-7
    assert abs(orc.lattice_sum(dim, 1.3) - float(total)) < 1e-14
