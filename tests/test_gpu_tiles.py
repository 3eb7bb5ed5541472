"""The FP32 density pass on cell-blocked shared-memory tiles against the
row walk over global memory (sph_params.pair_tiles = 0).  pair_tiles = 1,
one thread per particle over the tile, visits the same candidates in the
same order with the same arithmetic, so every state field after several
steps is bit for bit the same; so does pair_tiles = 3, the same walk with
each lane's rows taken as one sequence.  (Both hold whole cells: bit for
bit with a sort that does not refine the cells, x_subcells = 1; with the
default sub-cells the row walk cuts its runs finer, so the tiles add more
zero terms to the compensated sums and agree to FP32 rounding.)  pair_tiles = 2, groups of lanes sharing a
particle's candidates, writes the same neighbour lists but sums sigma in
another order: its densities agree to FP32 rounding, and it is checked
against the FP64 oracle like the other FP32 paths.  Cases: partial edge
blocks, halos that wrap a periodic axis more than once (5 cells per axis),
walls in a non-periodic box, the dual-criteria integrator (which freezes the
density pass's neighbour list for its substeps), and a block whose halo
exceeds the tile (its particles take the row walk inside the tile kernel)."""
import numpy as np
import pytest

import paper_2411_13992_gb300 as sph
from paper_2411_13992_gb300 import cases

from gpu_helpers import compare_step, oracle_trajectory

pytestmark = pytest.mark.gpu

FIELDS = ("x", "v", "a", "dr", "rho")


def _run(c, tiles, steps, **kw):
    sim = sph.Simulation(c, precision=32, pair_tiles=tiles, **kw)
    try:
        sim.set_state()
        sim.build_cells()
        sim.step(steps)
        assert sim.sync() is None
        return sim.get_state(), sim.diag()
    finally:
        sim.close()


def _clustered_tgv3d(n, count, seed=11):
    """3-D Taylor-Green lattice with ``count`` particles moved into a cube of
    2 x 2 x 2 cells, so that one block's halo holds several times the
    particles of the others (more than the tile holds)."""
    c = cases.tgv3d(n)
    x = c["x"].copy()
    edge = c["L"][0] / np.floor(c["L"][0] / c["h_max"])
    u = np.stack([cases.uniform(np.arange(count), k, seed) for k in range(3)], axis=1)
    x[:count] = (5.0 + 2.0 * u) * edge
    c = dict(c)
    c["x"] = x
    return c


CASES = {
    "tgv3d_24_partial_blocks": lambda: cases.tgv3d(24),
    "tgv3d_20": lambda: cases.tgv3d(20),
    "tgv3d_7_five_cells_per_axis": lambda: cases.tgv3d(7),
    "tgv2d_50": lambda: cases.tgv2d(50),
    "tgv2d_7_five_cells_per_axis": lambda: cases.tgv2d(7),
    "cavity2d_48_walls": lambda: cases.cavity2d(48),
    "tgv3d_24_halo_beyond_tile": lambda: _clustered_tgv3d(24, 2500),
}


@pytest.mark.parametrize("mode", [1, 3])
@pytest.mark.parametrize("name", sorted(CASES))
def test_tiled_walk_is_bit_identical_to_the_row_walk(name, mode):
    c = CASES[name]()
    got, d_got = _run(c, mode, 5, x_subcells=1)
    ref, d_ref = _run(c, 0, 5, x_subcells=1)
    for k in FIELDS:
        assert np.array_equal(got[k], ref[k]), (name, k)
    assert d_got["ke"] == d_ref["ke"]


@pytest.mark.parametrize("mode", [1, 3])
@pytest.mark.parametrize("name", ["tgv3d_24_partial_blocks", "tgv3d_7_five_cells_per_axis", "cavity2d_48_walls"])
def test_tiled_walk_matches_the_sub_cell_row_walk(name, mode):
    """With the default sub-cell sort the tiles walk whole cells and the row
    walk sub-cells: the same pairs, densities within FP32 rounding."""
    c = CASES[name]()
    fl = c["kind"] == 0
    got, _ = _run(c, mode, 0)
    ref, _ = _run(c, 0, 0)
    d_rho = np.abs(got["rho"][fl] - ref["rho"][fl]).max() / np.abs(ref["rho"][fl]).max()
    assert d_rho <= 2e-7, (name, d_rho)


@pytest.mark.parametrize("mode", [1, 3])
def test_tiled_density_is_bit_identical_in_the_dual_criteria_integrator(mode):
    c = cases.tgv3d(20)
    got, d_got = _run(c, mode, 3, integrator=sph.INT_DUAL, x_subcells=1)
    ref, d_ref = _run(c, 0, 3, integrator=sph.INT_DUAL, x_subcells=1)
    for k in ("x", "v", "rho"):
        assert np.array_equal(got[k], ref[k]), k
    assert d_got["substeps"] == d_ref["substeps"]


@pytest.mark.parametrize("name", sorted(CASES))
def test_cooperative_density_matches_the_row_walk(name):
    """From the same state (the initial force pass of sph_build_cells), the
    cooperative pass's densities equal the row walk's to FP32 rounding of a
    compensated sum of ~81 terms; after 5 steps the trajectories agree to the
    FP32 per-step bound."""
    c = CASES[name]()
    fl = c["kind"] == 0
    for steps in (0, 5):
        got, _ = _run(c, 2, steps)
        ref, _ = _run(c, 0, steps)
        assert np.isfinite(got["rho"]).all()
        d_rho = np.abs(got["rho"][fl] - ref["rho"][fl]).max() / np.abs(ref["rho"][fl]).max()
        assert d_rho <= (2e-7 if steps == 0 else 1e-5), (name, steps, d_rho)
        if steps:
            d_v = np.linalg.norm(got["v"][fl] - ref["v"][fl], axis=1).max() / np.linalg.norm(ref["v"][fl], axis=1).max()
            assert d_v <= 1e-5, (name, d_v)


@pytest.mark.parametrize("kind", ["tgv3d_16", "tgv3d_15", "cavity2d_32", "tgv2d_50"])
def test_cooperative_density_step_parity_with_the_oracle(kind):
    """One FP32 step from the oracle's state with pair_tiles = 2: the FP32
    bounds of the parity tests (1e-5 on x, v, rho, KE; 1e-3 on a and dr)."""
    c = {"tgv3d_16": lambda: cases.tgv3d(16), "tgv3d_15": lambda: cases.tgv3d(15),
         "cavity2d_32": lambda: cases.cavity2d(32, U=1.0), "tgv2d_50": lambda: cases.tgv2d(50)}[kind]()
    dt, states, P, s0 = oracle_trajectory(c, 3, {0, 3})
    for k in (0, 3):
        err, _, _ = compare_step(c, states[k], dt, s0, P, precision=32, pair_tiles=2)
        for f in ("x", "v", "rho", "ke"):
            assert err[f] <= 1e-5, (kind, k, f, err)
        assert err["a"] <= 1e-3, (kind, k, err)
        if err["n_chi_ref"]:
            assert err["dr"] <= 1e-3, (kind, k, err)
