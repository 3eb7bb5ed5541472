"""A context given a new state behaves as a fresh one.

The sort leaves h, m, sigma0 and kind in place while they are alike for all
particles (both state sets then hold them), so a state set after steps on
another state must refresh both sets: uniform masses of another value, masses
that vary over the particles, and uniform masses again.  After each new state
and a few steps the context's state is bit for bit that of a fresh context
given the same state, in both precisions."""
import numpy as np
import pytest

import paper_2411_13992_gb300 as sph
from paper_2411_13992_gb300 import cases

pytestmark = pytest.mark.gpu

FIELDS = ("x", "v", "a", "dr", "rho")


def _run(sim, steps):
    sim.set_state()
    sim.build_cells()
    sim.step(steps)
    assert sim.sync() is None
    return sim.get_state()


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("make", [lambda: cases.tgv3d(12), lambda: cases.tgv2d(40)], ids=["tgv3d_12", "tgv2d_40"])
def test_new_state_on_a_used_context_matches_a_fresh_context(make, precision):
    base = make()
    n = base["n"]
    m0 = np.asarray(base["m"], dtype=np.float64)
    ramp = 1.0 + 0.02 * (np.arange(n) % 7) / 7.0
    masses = [m0 * 1.1, m0 * ramp, m0]   # uniform (another value), varying, uniform again
    sim = sph.Simulation(dict(base), precision=precision)
    try:
        _run(sim, 3)
        for m in masses:
            c = dict(base)
            c["m"] = np.ascontiguousarray(m)
            sim.case = c
            got = _run(sim, 3)
            fresh = sph.Simulation(dict(c), precision=precision)
            try:
                ref = _run(fresh, 3)
            finally:
                fresh.close()
            for k in FIELDS:
                assert np.array_equal(got[k], ref[k]), (k, precision)
    finally:
        sim.close()
