"""The largest particle count the library takes: n <= 2^25 (a neighbour-list
entry holds j in 25 bits beside a 7-bit stencil code).

A 2-D Taylor-Green vortex of 5792^2 = 33,547,264 particles (FP32 form):
* the densities of sampled particles against the oracle evaluated on each
  sample's own neighbourhood (the 7 x 7 lattice block around it holds every
  particle within 2h = 2.6 dp of it: jitter is 1e-3 dp);
* two kick-drift-kick steps keep the mass exactly, the momentum to rounding,
  lower the kinetic energy and raise no device error.
One particle more than 2^25 is refused on the host (tests/test_abi_cpu.py)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2411_13992_gb300 as sph
from paper_2411_13992_gb300 import cases

from gpu_helpers import oracle_params

pytestmark = pytest.mark.gpu

SIDE = 5792


def test_maximum_particle_count():
    assert torch.cuda.is_available()
    c = cases.tgv2d(SIDE)
    n = c["n"]
    assert n <= 2 ** 25 and n > 2 ** 25 - 8192
    sim = sph.Simulation(c, precision=32)
    try:
        sim.set_state()
        sim.build_cells()
        rho = np.zeros(n)
        sph.sph_get_state(sim.ctx, None, None, None, None, rho)
        d0 = sim.diag()
        sim.step(2)
        assert sim.sync() is None
        d1 = sim.diag()
    finally:
        sim.close()
    # sampled densities against the oracle on local neighbourhoods
    P = oracle_params(c)
    rng = np.random.default_rng(7)
    offs = np.arange(-3, 4)
    worst = 0.0
    for s in rng.integers(0, n, 40):
        ix, iy = s % SIDE, s // SIDE
        bx, by = np.meshgrid((ix + offs) % SIDE, (iy + offs) % SIDE, indexing="ij")
        ids = (bx + SIDE * by).ravel()
        sub = {k: np.ascontiguousarray(c[k][ids]) for k in ("x", "h", "m", "kind")}
        me = int(np.nonzero(ids == s)[0][0])
        s0 = oracle.sigma0_for({"h": sub["h"], "m": sub["m"], "rho0": c["rho0"]}, 2)
        nb = oracle.neighbours(P, sub["x"], sub["h"], "brute")
        ref, _ = oracle.density(P, sub["x"], sub["h"], sub["kind"], s0, nb)
        worst = max(worst, abs(rho[s] - ref[me]) / ref[me])
    print("n = %d: worst sampled density error %.2e; KE %.6g -> %.6g" % (n, worst, d0["ke"], d1["ke"]))
    assert worst < 1e-6
    assert d1["mass"] == d0["mass"] and d1["steps"] == 2
    assert np.abs(d1["momentum"] - d0["momentum"]).max() < 1e-5 * d0["mass"] * d0["vmax"]
    assert 0.0 < d1["ke"] < d0["ke"]
