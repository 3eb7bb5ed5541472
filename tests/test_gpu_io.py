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


def test_save_ckpt_writes_the_state_the_adjoint_replays_from():
    """sph_save_ckpt writes x, v, a, dr as sph_get_state does, with the next
    step size and the step count of sph_get_diag; an adjoint segment replayed
    from it equals one replayed from sph_get_state's arrays."""
    import torch
    from paper_2411_13992_gb300 import cases
    c = cases.tgv2d(24)
    sim = sph.Simulation(c, precision=64, fixed_dt=1.0e-3, adjoint_steps=3)
    try:
        sim.set_state()
        sim.build_cells()
        sim.step(4)
        n = c["n"]
        ck = {k: np.zeros((n, 3)) for k in ("x", "v", "a", "dr")}
        dt_next, steps = sph.sph_save_ckpt(sim.ctx, ck["x"], ck["v"], ck["a"], ck["dr"])
        st = sim.get_state()
        for k in ("x", "v", "a", "dr"):
            assert np.array_equal(ck[k], st[k]), k
        d = sim.diag()
        assert dt_next == d["dt_next"] and steps == d["steps"] == 4
        # device destinations too
        dev = {k: torch.zeros((n, 3), dtype=torch.float64, device=sim.device) for k in ck}
        sph.sph_save_ckpt(sim.ctx, dev["x"], dev["v"], dev["a"], dev["dr"])
        for k in ck:
            assert np.array_equal(dev[k].cpu().numpy(), ck[k]), k
        outs = []
        for src in (ck, st):
            xb, vb = np.ones((n, 3)), np.zeros((n, 3))
            ab, drb = np.zeros((n, 3)), np.zeros((n, 3))
            eb = sph.sph_step_adjoint(sim.ctx, src["x"], src["v"], src["a"], src["dr"], 3, xb, vb, ab, drb)
            outs.append((xb, vb, eb))
        assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    finally:
        sim.close()
