"""Pins of the oracle's pair sums by exact symmetries: pairwise momentum
conservation of Eq. 3 + Eq. 7 (antisymmetric pair terms), angular momentum
of the pressure force (central pair terms), Galilean and translation
invariance, and identical neighbour sets from brute force and cells.  A term
that uses rho_i^2 for rho_i rho_j, an unsymmetric P*, or a non-central
pressure direction breaks one of these to O(1)."""
import numpy as np
import pytest

from paper_2411_13992_gb300 import cases


def _random_state(orc, dim, n, seed, periodic=True, jit=0.15, var_h=True, eta=0.02, vamp=3.0):
    c = cases.lattice_block(dim, n, dp=0.1, periodic=periodic, jitter_dp=jit, seed=seed)
    rng = np.random.default_rng(seed)
    N = c["n"]
    if var_h:
        c["h"] = c["h"] * rng.uniform(0.85, 1.15, N)
    c["m"] = c["m"] * rng.uniform(0.9, 1.1, N)
    v = np.zeros((N, 3))
    v[:, :dim] = rng.uniform(-vamp, vamp, (N, dim))     # |dU|/c spans beta < 1 and beta = 1
    P = orc.make_params(dim, c["lo"], c["L"], c["periodic"], 1.0, 10.0, eta, float(c["h"].min()),
                        tv_mode=2)
    nb = orc.neighbours(P, c["x"], c["h"], "cells")
    s0 = np.full(N, orc.lattice_sum(dim, 1.3) / 0.1 ** dim)
    rho, _ = orc.density(P, c["x"], c["h"], c["kind"], s0, nb)
    return c, P, v, nb, rho


@pytest.mark.parametrize("dim,n", [(2, 14), (3, 7)])
@pytest.mark.parametrize("h_pair_max", [False, True])
def test_total_momentum_is_conserved(orc, dim, n, h_pair_max):
    c, P, v, nb, rho = _random_state(orc, dim, n, seed=11 + dim)
    P.h_pair_max = int(h_pair_max)
    nb = orc.neighbours(P, c["x"], c["h"], "cells")
    f = orc.forces(P, c["x"], v, c["h"], c["m"], c["kind"], c["vw"], rho, nb)
    mom = (c["m"][:, None] * f["a"]).sum(axis=0)
    scale = (c["m"][:, None] * np.abs(f["a"])).sum()
    assert scale > 0
    assert np.abs(mom).max() < 1e-13 * scale, (mom, scale)
    # sanity: both the Riemann dissipation and the viscous term were active
    assert 2.0 * np.abs(v).max() / P.c > 1.0 / 3.0     # pairs with dU/c > 1/3 exist


@pytest.mark.parametrize("dim,n", [(2, 12), (3, 6)])
def test_pressure_force_conserves_angular_momentum(orc, dim, n):
    c, P, v, nb, rho = _random_state(orc, dim, n, seed=5, periodic=False, eta=0.0)
    f = orc.forces(P, c["x"], v, c["h"], c["m"], c["kind"], c["vw"], rho, nb)
    ma = c["m"][:, None] * f["a"]
    Lz = np.cross(c["x"], ma).sum(axis=0)
    scale = (np.linalg.norm(c["x"], axis=1) * np.linalg.norm(ma, axis=1)).sum()
    assert np.abs(Lz).max() < 1e-13 * scale


@pytest.mark.parametrize("dim,n", [(2, 12), (3, 6)])
def test_galilean_invariance(orc, dim, n):
    c, P, v, nb, rho = _random_state(orc, dim, n, seed=7)
    f0 = orc.forces(P, c["x"], v, c["h"], c["m"], c["kind"], c["vw"], rho, nb)
    shift = np.zeros(3)
    shift[:dim] = [0.75, -1.25, 0.5][:dim]
    f1 = orc.forces(P, c["x"], v + shift, c["h"], c["m"], c["kind"], c["vw"], rho, nb)
    for k in ("a", "R", "dr"):
        np.testing.assert_allclose(f1[k], f0[k], rtol=0, atol=1e-12 * np.abs(f0[k]).max())


@pytest.mark.parametrize("dim,n", [(2, 12), (3, 6)])
def test_translation_invariance_periodic(orc, dim, n):
    c, P, v, nb, _ = _random_state(orc, dim, n, seed=9)
    s0 = np.full(c["n"], orc.lattice_sum(dim, 1.3) / 0.1 ** dim)
    case = dict(c)
    out0 = orc.force_pass(P, case, c["x"], v, s0)
    x1 = c["x"].copy()
    for d in range(dim):
        x1[:, d] = np.mod(x1[:, d] + 0.3719 * c["L"][d], c["L"][d])
    out1 = orc.force_pass(P, case, x1, v, s0)
    np.testing.assert_allclose(out1["rho"], out0["rho"], rtol=1e-11)
    for k in ("a", "R"):
        np.testing.assert_allclose(out1[k], out0[k], rtol=0, atol=1e-9 * np.abs(out0[k]).max())


@pytest.mark.parametrize("dim,n,periodic", [(2, 13, True), (2, 11, False), (3, 7, True), (3, 6, False)])
def test_cells_and_brute_force_find_the_same_neighbours(orc, dim, n, periodic):
    c, P, v, _, _ = _random_state(orc, dim, n, seed=3, periodic=periodic)
    s_b, i_b = orc.neighbours(P, c["x"], c["h"], "brute")
    s_c, i_c = orc.neighbours(P, c["x"], c["h"], "cells")
    np.testing.assert_array_equal(s_b, s_c)
    np.testing.assert_array_equal(i_b, i_c)
    # every listed pair is within 2 h_ij, self included exactly once
    assert all(i in i_b[s_b[i]:s_b[i + 1]] for i in range(c["n"]))
