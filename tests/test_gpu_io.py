"""State transfer through the C ABI: sph_set_state reads the caller's rows in
place when the device can reach them (page-locked host memory, device
memory) and through the staging buffer otherwise (pageable host memory);
sph_get_state gathers the rows in the caller's order.  Every source and
destination kind gives the same state bit for bit."""
import numpy as np
import pytest
import torch

import paper_2411_13992_gb300 as sph
from paper_2411_13992_gb300 import cases

pytestmark = pytest.mark.gpu


def _run(c, precision, kind):
    n = c["n"]
    host = {k: np.ascontiguousarray(c[k]) for k in ("x", "v")}
    if kind == "pageable":
        src = host
    elif kind == "pinned":
        src = {k: torch.from_numpy(host[k]).pin_memory() for k in host}
    else:
        src = {k: torch.from_numpy(host[k]).cuda() for k in host}
    sim = sph.Simulation(c, precision=precision)
    try:
        sph.sph_set_state(sim.ctx, src["x"], src["v"], None, None, c["h"], c["m"], c.get("kind"), c.get("vw"),
                          None)
        sim.build_cells()
        sim.step(3)
        out = {}
        for dest in ("pageable", "pinned", "device"):
            if dest == "pageable":
                o = {k: np.zeros((n, 3)) for k in ("x", "v", "a", "dr")}
                o["rho"] = np.zeros(n)
            elif dest == "pinned":
                o = {k: torch.zeros((n, 3), dtype=torch.float64).pin_memory() for k in ("x", "v", "a", "dr")}
                o["rho"] = torch.zeros(n, dtype=torch.float64).pin_memory()
            else:
                o = {k: torch.zeros((n, 3), dtype=torch.float64, device="cuda") for k in ("x", "v", "a", "dr")}
                o["rho"] = torch.zeros(n, dtype=torch.float64, device="cuda")
            sph.sph_get_state(sim.ctx, o["x"], o["v"], o["a"], o["dr"], o["rho"])
            torch.cuda.synchronize()
            out[dest] = {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in o.items()}
        assert sim.sync() is None
        return out
    finally:
        sim.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_every_source_and_destination_gives_the_same_state(precision):
    c = cases.cavity2d(24, U=1.0, jitter_dp=0.05, seed=9)
    runs = {kind: _run(c, precision, kind) for kind in ("pageable", "pinned", "device")}
    ref = runs["pageable"]["pageable"]
    for kind, out in runs.items():
        for dest, st in out.items():
            for k in ("x", "v", "a", "dr", "rho"):
                assert np.array_equal(st[k], ref[k]), (kind, dest, k)
    # rows come back in the caller's order: particle k's position moved by less than a cell
    assert np.abs(ref["x"] - c["x"]).max() < c["h_max"]
