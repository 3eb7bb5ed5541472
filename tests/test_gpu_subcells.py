"""The sub-cell cut of the row walks (sph_params.x_subcells): the counting
sort refines each cell along x into 2 or 4 sub-cells (ordered by sub-cell,
then by id, within the cell) and the density passes cut each row's x extent
at sub-cell rather than cell granularity.  The accepted neighbours must stay
those of the full 5^D stencil (Eq. 8 sums over every j with r < 2h).

Isolated particle pairs make a dropped neighbour visible: each pair's
particles lie at r = 2h (1 - delta) from each other and more than 2h from
every other particle, so each density is W(0) + W(r) of one term each, which
the oracle computes with brute-force neighbours.  delta down to 2e-3 puts
W(r) / W(0) at ~1e-11, which the FP64 form resolves (the FP64 density pass
takes its candidates from the same FP32 row walk); a third of the pairs lie
along x, the axis the cut works on, the others in random directions; every
pair is shifted by one random offset so that some straddle the periodic
boundary, and one layout has walls of the box along x instead.  Then whole
steps of the generated workloads at x_subcells 1, 2 and 4: the same
neighbours summed in another order, so the states agree to rounding."""
import math

import numpy as np
import pytest

import oracle
import paper_2411_13992_gb300 as sph
from paper_2411_13992_gb300 import cases

from gpu_helpers import normwise, oracle_params

pytestmark = pytest.mark.gpu


def _isolated_pairs(dim, nb, delta_lo, delta_hi, periodic_x=True, seed=7):
    """nb^dim blocks of side 8h, one pair per block (centre within h of the
    block centre, separation 2h (1 - delta)); h = 1, dp = 1."""
    h = 1.0
    B = 8.0 * h
    L = nb * B
    nblk = nb ** dim
    ids = np.arange(nblk)
    u = np.stack([cases.uniform(ids, k, seed) for k in range(4)], axis=1)
    grid = np.stack(np.meshgrid(*[np.arange(nb)] * dim, indexing="ij"), axis=-1).reshape(-1, dim)
    centre = np.zeros((nblk, 3))
    centre[:, :dim] = (grid + 0.5) * B + (2.0 * u[:, :dim] - 1.0) * h
    # directions: along +-x for a third, random otherwise
    dirs = np.zeros((nblk, 3))
    g = np.stack([cases.uniform(ids, k, seed + 1) for k in range(3)], axis=1)
    if dim == 2:
        ang = 2 * math.pi * g[:, 0]
        dirs[:, 0], dirs[:, 1] = np.cos(ang), np.sin(ang)
    else:
        z = 2 * g[:, 0] - 1
        ang = 2 * math.pi * g[:, 1]
        s = np.sqrt(1 - z * z)
        dirs[:, 0], dirs[:, 1], dirs[:, 2] = s * np.cos(ang), s * np.sin(ang), z
    along_x = ids % 3 == 0
    dirs[along_x] = 0.0
    dirs[along_x, 0] = np.where(g[along_x, 2] < 0.5, -1.0, 1.0)
    delta = delta_lo * (delta_hi / delta_lo) ** u[:, 3]
    r = 2.0 * h * (1.0 - delta)
    x = np.concatenate([centre - 0.5 * r[:, None] * dirs, centre + 0.5 * r[:, None] * dirs])
    periodic = [1] * dim + [0] * (3 - dim)
    if periodic_x:
        off = np.zeros(3)
        off[:dim] = (2.0 * cases.uniform(np.arange(dim), 0, seed + 2) + 0.5) * h
        x[:, :dim] = np.mod(x[:, :dim] + off[:dim], L)
    else:
        periodic[0] = 0
    Ls = (L, L, L if dim == 3 else 1.0)
    return cases._case("isolated_pairs", dim, (0, 0, 0), Ls, periodic, 1.0, 10.0, 0.01, 1.0, x,
                       np.zeros_like(x), h, 1.0)


def _density(c, precision, xs):
    sim = sph.Simulation(c, precision=precision, x_subcells=xs)
    try:
        sim.set_state()
        sim.build_cells()
        assert sim.sync() is None
        return sim.get_state()["rho"]
    finally:
        sim.close()


def _oracle_density(c):
    P = oracle_params(c)
    s0 = oracle.sigma0_for(c, c["dim"])
    nb = oracle.neighbours(P, c["x"], c["h"], mode="brute")
    # every particle has itself and its partner
    assert np.all(np.diff(nb[0]) == 2)
    rho, _ = oracle.density(P, c["x"], c["h"], c["kind"], s0, nb)
    return rho


@pytest.mark.parametrize("xs", [1, 2, 4])
@pytest.mark.parametrize("dim,nb,periodic_x", [(2, 12, True), (3, 6, True), (3, 6, False), (2, 12, False)])
def test_pairs_at_the_support_edge_fp64(dim, nb, periodic_x, xs):
    c = _isolated_pairs(dim, nb, 2e-3, 0.3, periodic_x)
    want = _oracle_density(c)
    got = _density(c, 64, xs)
    # a dropped partner would move rho by W(r)/W(0) >= ~1e-11 of rho
    rel = np.abs(got - want) / np.abs(want)
    assert rel.max() <= 1e-13, (dim, xs, rel.max(), int(np.argmax(rel)))


@pytest.mark.parametrize("xs", [1, 4])
@pytest.mark.parametrize("dim,nb,periodic_x", [(2, 12, True), (3, 6, True), (3, 6, False)])
def test_pairs_at_the_support_edge_fp32(dim, nb, periodic_x, xs):
    c = _isolated_pairs(dim, nb, 0.05, 0.3, periodic_x)
    want = _oracle_density(c)
    got = _density(c, 32, xs)
    # W(r)/W(0) >= 3e-5 here: far above the FP32 form's ~1e-7
    rel = np.abs(got - want) / np.abs(want)
    assert rel.max() <= 2e-6, (dim, xs, rel.max())


WORKLOADS = {
    "tgv3d_24": lambda: cases.tgv3d(24),
    "tgv3d_7_five_cells_per_axis": lambda: cases.tgv3d(7),
    "tgv2d_50": lambda: cases.tgv2d(50),
    "cavity2d_48_walls": lambda: cases.cavity2d(48),
    "cylinder2d_variable_h": lambda: cases.cylinder2d(res=6),
}


def _disp(x, c):
    """Displacement from the initial positions, minimum image on periodic axes."""
    d = x - c["x"]
    for k in range(c["dim"]):
        if c["periodic"][k]:
            d[:, k] -= c["L"][k] * np.round(d[:, k] / c["L"][k])
    return d


def _steps(c, precision, xs, steps):
    sim = sph.Simulation(c, precision=precision, x_subcells=xs)
    try:
        sim.set_state()
        sim.build_cells()
        sim.step(steps)
        assert sim.sync() is None
        return sim.get_state(), sim.diag()
    finally:
        sim.close()


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_steps_agree_across_sub_cell_counts(name, precision):
    """Five steps at x_subcells 1, 2 and 4 from the same state: the same
    neighbours in another summation order, within the per-step bounds of the
    parity tests (FP64 1e-12, FP32 1e-5 on x, v, rho; the displacement of x,
    whose relative rounding is largest where the pressure terms nearly cancel,
    as in the cavity at rest)."""
    c = WORKLOADS[name]()
    fl = c["kind"] == 0
    ref, d_ref = _steps(c, precision, 1, 5)
    tol = 1e-12 if precision == 64 else 1e-5
    for xs in (2, 4):
        got, d_got = _steps(c, precision, xs, 5)
        for k in ("x", "v", "rho"):
            if k == "x":
                err = normwise(_disp(got[k], c)[fl], _disp(ref[k], c)[fl])
            else:
                err = normwise(got[k][fl], ref[k][fl])
            assert err <= tol, (name, precision, xs, k, err)
        assert abs(d_got["ke"] - d_ref["ke"]) <= tol * abs(d_ref["ke"])
