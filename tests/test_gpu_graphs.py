"""CUDA graph replay of kick-drift-kick steps (sph_params.graphs): the
replayed steps give bit-identical states to directly launched ones (odd step
counts, both precisions, walls, a viscosity change between calls), count the
same kernel launches, and run faster where launches dominate (2,500
particles)."""
import time

import numpy as np
import pytest
import torch

import paper_2411_13992_gb300 as sph
from paper_2411_13992_gb300 import cases

pytestmark = pytest.mark.gpu


def _run(c, precision, graphs, plan):
    sim = sph.Simulation(c, precision=precision, graphs=graphs)
    try:
        sim.set_state()
        sim.build_cells()
        l0 = sim.launches()
        for what, arg in plan:
            if what == "step":
                sim.step(arg)
            else:
                sph.sph_set_eta(sim.ctx, arg)
        assert sim.sync() is None
        return sim.get_state(), sim.diag(), sim.launches() - l0
    finally:
        sim.close()


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("kind", ["tgv", "cavity"])
def test_graph_replay_is_bit_identical(precision, kind):
    c = cases.tgv2d(50) if kind == "tgv" else cases.cavity2d(40)
    plan = [("step", 7), ("step", 1), ("eta", 2.0 * c["eta"]), ("step", 10), ("step", 3)]
    g_on, d_on, l_on = _run(c, precision, 1, plan)
    g_off, d_off, l_off = _run(c, precision, 0, plan)
    for k in ("x", "v", "a", "dr", "rho"):
        assert np.array_equal(g_on[k], g_off[k]), k
    assert d_on["ke"] == d_off["ke"] and d_on["steps"] == d_off["steps"] == 21
    assert l_on == l_off


def test_graph_replay_is_faster_for_small_cases():
    c = cases.tgv2d(50)
    times = {}
    for graphs in (0, 1):
        sim = sph.Simulation(c, precision=64, graphs=graphs)
        try:
            sim.set_state()
            sim.build_cells()
            sim.step(20)
            sim.sync()
            t0 = time.perf_counter()
            sim.step(400)
            sim.sync()
            times[graphs] = (time.perf_counter() - t0) / 400 * 1e3
        finally:
            sim.close()
    print("2-D Taylor-Green 50^2 FP64: %.1f us per step launched directly, %.1f us replayed from graphs"
          % (times[0] * 1e3, times[1] * 1e3))
    assert times[1] < times[0]


def _adjoint_run(c, precision, graphs, plan):
    """sph_step_adjoint called per plan entry (segment length, eta or None)
    from the same checkpoint; returns every call's cotangents."""
    dt = 0.5 * 0.25 * c["h_min"] / 10.0
    sim = sph.Simulation(c, precision=precision, graphs=graphs, fixed_dt=dt, adjoint_steps=6)
    out = []
    try:
        sim.set_state()
        sim.build_cells()
        s0 = sim.get_state()
        rng = np.random.default_rng(5)
        n = c["n"]
        for T, eta in plan:
            if eta is not None:
                sph.sph_set_eta(sim.ctx, eta)
            w = [np.ascontiguousarray(np.pad(rng.standard_normal((n, 2)), ((0, 0), (0, 1)))) for _ in range(4)]
            eb = sph.sph_step_adjoint(sim.ctx, s0["x"], s0["v"], s0["a"], s0["dr"], T, *w)
            out.append((w, eb))
        assert sim.sync() is None
        return out, sim.launches()
    finally:
        sim.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_adjoint_segment_replay_is_bit_identical(precision):
    """The adjoint's segment (forward replay with the tape, reverse sweep)
    replayed from a graph gives the same cotangents bit for bit as launched
    directly: repeated segments, a change of segment length (recapture), and
    a viscosity change between calls (the graph is released)."""
    c = cases.tgv2d(24, jitter_dp=0.05, seed=4)
    plan = [(6, None), (6, None), (3, None), (6, 2.0 * c["eta"]), (6, None)]
    on, l_on = _adjoint_run(c, precision, 1, plan)
    off, l_off = _adjoint_run(c, precision, 0, plan)
    for (w1, e1), (w0, e0) in zip(on, off):
        for a, b in zip(w1, w0):
            assert np.array_equal(a, b)
        assert e1 == e0
    assert l_on == l_off
