"""Seeded synthetic particle layouts for the WCSPH transport-velocity step.

This module only lays out particles: lattice positions, a counter-based
jitter, the initial velocity fields of the test flows, masses, smoothing
lengths, particle kinds and wall velocities.  It holds none of the method's
arithmetic (no kernel, density, force or time-step formula), so both the CUDA
library's callers and the FP64 oracle may take their inputs from it.

Jitter: uniform in [-amp, amp) * dp per component, drawn from splitmix64 of
(seed, particle id, component) -- a counter-based generator, so any subset of
particles can be regenerated independently.

Cases (Sec. 4 of the paper and the workloads derived from it):

* ``tgv2d``  -- 2-D Taylor-Green vortex on the periodic unit square
  (Sec. 4.1), u = sin(2 pi x) cos(2 pi y), v = -cos(2 pi x) sin(2 pi y).
* ``tgv3d``  -- 3-D Taylor-Green vortex on the periodic box [0, 2 pi]^3,
  u = sin x cos y cos z, v = -cos x sin y cos z, w = 0 (not in the paper).
* ``cavity2d`` -- 2-D lid-driven cavity, unit square with three layers of
  wall particles, lid velocity (U, 0) (Sec. 4.2 geometry).
* ``cylinder2d`` -- variable-resolution layout around a cylinder: a coarse far
  field, a refinement rectangle at half the spacing, and a smooth smoothing
  length blend in a band outside the rectangle (Sec. 4.4 layout).
"""
from __future__ import annotations

import math

import numpy as np

SEED = 20241121
H_OVER_DP = 1.3          # h = 1.3 dp (Sec. 4)

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(counter: np.ndarray, seed: int) -> np.ndarray:
    """splitmix64 output for each 64-bit counter under ``seed``."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (counter.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(ids: np.ndarray, comp: int, seed: int) -> np.ndarray:
    """Uniform [0, 1) doubles for (particle id, component)."""
    ctr = ids.astype(np.uint64) * np.uint64(4) + np.uint64(comp)
    return (splitmix64(ctr, seed) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def jitter(ids: np.ndarray, dim: int, amp_dp: float, seed: int) -> np.ndarray:
    """(N, 3) displacements uniform in [-amp_dp, amp_dp) along the first dim axes."""
    out = np.zeros((len(ids), 3))
    for d in range(dim):
        out[:, d] = (2.0 * uniform(ids, d, seed) - 1.0) * amp_dp
    return out


def _lattice(counts, dp, origin):
    axes = [origin[d] + (np.arange(counts[d]) + 0.5) * dp for d in range(len(counts))]
    grids = np.meshgrid(*axes, indexing="ij")
    pts = np.stack([g.ravel(order="F") for g in grids], axis=1)
    out = np.zeros((len(pts), 3))
    out[:, : len(counts)] = pts
    return out


def _case(name, dim, lo, L, periodic, rho0, c, eta, u_ref, x, v, h, m, kind=None, vw=None, g=(0.0, 0.0, 0.0),
          **extra):
    n = len(x)
    h = np.ascontiguousarray(np.broadcast_to(np.asarray(h, np.float64), (n,)))
    m = np.ascontiguousarray(np.broadcast_to(np.asarray(m, np.float64), (n,)))
    kind = np.zeros(n, np.int8) if kind is None else np.asarray(kind, np.int8)
    vw = np.zeros((n, 3)) if vw is None else np.asarray(vw, np.float64)
    fluid = kind == 0
    d = dict(name=name, dim=dim, lo=tuple(float(t) for t in lo), L=tuple(float(t) for t in L),
             periodic=tuple(int(t) for t in periodic), rho0=float(rho0), c=float(c), eta=float(eta),
             u_ref=float(u_ref), g=tuple(float(t) for t in g),
             x=np.ascontiguousarray(x), v=np.ascontiguousarray(v), h=h, m=m, kind=kind, vw=vw,
             h_min=float(h[fluid].min() if fluid.any() else h.min()), h_max=float(h.max()), n=n)
    d.update(extra)
    return d


def tgv2d(n: int = 50, Re: float = 100.0, U: float = 1.0, c0: float = 10.0, rho0: float = 1.0,
          jitter_dp: float = 1.0e-3, seed: int = SEED):
    """2-D Taylor-Green vortex, periodic [0,1]^2, n x n particles at (k+1/2) dp
    plus jitter; nu = U L / Re with L = 1."""
    dp = 1.0 / n
    x = _lattice((n, n), dp, (0.0, 0.0))
    ids = np.arange(len(x))
    x += jitter(ids, 2, jitter_dp * dp, seed)
    v = np.zeros_like(x)
    v[:, 0] = U * np.sin(2 * math.pi * x[:, 0]) * np.cos(2 * math.pi * x[:, 1])
    v[:, 1] = -U * np.cos(2 * math.pi * x[:, 0]) * np.sin(2 * math.pi * x[:, 1])
    nu = U * 1.0 / Re
    return _case("tgv2d", 2, (0, 0, 0), (1, 1, 1), (1, 1, 0), rho0, c0, rho0 * nu, U, x, v,
                 H_OVER_DP * dp, rho0 * dp ** 2, dp=dp, Re=Re, U=U, nu=nu, seed=seed)


def tgv3d(n: int = 128, Re: float = 1600.0, U: float = 1.0, c0: float = 10.0, rho0: float = 1.0,
          jitter_dp: float = 1.0e-3, seed: int = SEED):
    """3-D Taylor-Green vortex, periodic [0, 2 pi]^3, n^3 particles, nu = U L / Re
    with U = L = 1."""
    Lb = 2.0 * math.pi
    dp = Lb / n
    x = _lattice((n, n, n), dp, (0.0, 0.0, 0.0))
    ids = np.arange(len(x))
    x += jitter(ids, 3, jitter_dp * dp, seed)
    v = np.zeros_like(x)
    sx, cx = np.sin(x[:, 0]), np.cos(x[:, 0])
    sy, cy = np.sin(x[:, 1]), np.cos(x[:, 1])
    cz = np.cos(x[:, 2])
    v[:, 0] = U * sx * cy * cz
    v[:, 1] = -U * cx * sy * cz
    nu = U * 1.0 / Re
    return _case("tgv3d", 3, (0, 0, 0), (Lb, Lb, Lb), (1, 1, 1), rho0, c0, rho0 * nu, U, x, v,
                 H_OVER_DP * dp, rho0 * dp ** 3, dp=dp, Re=Re, U=U, nu=nu, seed=seed)


def cavity2d(n: int = 256, U: float = 1.0, Re: float = 100.0, layers: int = 3, rho0: float = 1.0,
             jitter_dp: float = 1.0e-3, seed: int = SEED):
    """2-D lid-driven cavity: n x n fluid particles in [0,1]^2 (jittered), wall
    particles on the lattice in ``layers`` rows around it; the top rows move
    with (U, 0).  c = 10 U, nu = U / Re."""
    dp = 1.0 / n
    tot = n + 2 * layers
    allp = _lattice((tot, tot), dp, (-layers * dp, -layers * dp))
    k = np.rint(allp[:, :2] / dp - 0.5).astype(np.int64)   # integer cell indices, fluid in [0, n)
    inside = (k[:, 0] >= 0) & (k[:, 0] < n) & (k[:, 1] >= 0) & (k[:, 1] < n)
    fluid = allp[inside]
    wall = allp[~inside]
    ids = np.arange(len(fluid))
    fluid = fluid + jitter(ids, 2, jitter_dp * dp, seed)
    x = np.concatenate([fluid, wall])
    kind = np.concatenate([np.zeros(len(fluid), np.int8), np.ones(len(wall), np.int8)])
    vw = np.zeros_like(x)
    lid = (kind == 1) & (x[:, 1] > 1.0)
    vw[lid, 0] = U
    v = np.zeros_like(x)
    nu = U / Re
    lo = (-layers * dp, -layers * dp, 0.0)
    L = (1.0 + 2 * layers * dp, 1.0 + 2 * layers * dp, 1.0)
    return _case("cavity2d", 2, lo, L, (0, 0, 0), rho0, 10.0 * U, rho0 * nu, U, x, v,
                 H_OVER_DP * dp, rho0 * dp ** 2, kind=kind, vw=vw, dp=dp, Re=Re, U=U, nu=nu, seed=seed,
                 n_fluid=len(fluid), n_wall=len(wall))


def cylinder2d(D: float = 1.0, res: int = 36, box=(30.0, 16.0), center=(10.0, 8.0),
               refine=(8.0, 24.0, 5.0, 11.0), band_dp: float = 4.0, layers: int = 3,
               U: float = 1.0, Re: float = 100.0, rho0: float = 1.0, c0: float = 10.0,
               jitter_dp: float = 1.0e-3, seed: int = SEED):
    """Variable-resolution layout: far field at dp = D/res, refinement
    rectangle [x0,x1]x[y0,y1] at dp/2, h blended linearly from 1.3 dp/2 to
    1.3 dp over ``band_dp`` coarse spacings outside the rectangle; a cylinder
    of diameter D made of ``layers`` rings of wall particles at the fine
    spacing; periodic box; uniform initial velocity (U, 0)."""
    dpc = D / res
    dpf = 0.5 * dpc
    x0, x1, y0, y1 = refine
    nx, ny = int(round(box[0] / dpc)), int(round(box[1] / dpc))
    coarse = _lattice((nx, ny), dpc, (0.0, 0.0))
    in_rect = (coarse[:, 0] > x0) & (coarse[:, 0] < x1) & (coarse[:, 1] > y0) & (coarse[:, 1] < y1)
    coarse = coarse[~in_rect]
    fx, fy = int(round((x1 - x0) / dpf)), int(round((y1 - y0) / dpf))
    fine = _lattice((fx, fy), dpf, (x0, y0))
    R = 0.5 * D
    def outside_cyl(p):
        return np.hypot(p[:, 0] - center[0], p[:, 1] - center[1]) >= R
    coarse = coarse[outside_cyl(coarse)]
    fine = fine[outside_cyl(fine)]
    rings = []
    for k in range(layers):
        rk = R - (k + 0.5) * dpf
        nk = max(int(round(2 * math.pi * rk / dpf)), 3)
        th = (np.arange(nk) + 0.5) * (2 * math.pi / nk)
        ring = np.zeros((nk, 3))
        ring[:, 0] = center[0] + rk * np.cos(th)
        ring[:, 1] = center[1] + rk * np.sin(th)
        rings.append(ring)
    wall = np.concatenate(rings)
    fluid = np.concatenate([fine, coarse])
    ids = np.arange(len(fluid))
    dp_f = np.concatenate([np.full(len(fine), dpf), np.full(len(coarse), dpc)])
    fluid = fluid + jitter(ids, 2, 1.0, seed) * (jitter_dp * dp_f)[:, None]
    # distance of coarse particles to the refinement rectangle -> h blend
    px, py = fluid[:, 0], fluid[:, 1]
    ddx = np.maximum(np.maximum(x0 - px, px - x1), 0.0)
    ddy = np.maximum(np.maximum(y0 - py, py - y1), 0.0)
    dist = np.hypot(ddx, ddy)
    t = np.clip(dist / (band_dp * dpc), 0.0, 1.0)
    h_f = np.where(dp_f == dpf, H_OVER_DP * dpf, H_OVER_DP * (dpf + t * (dpc - dpf)))
    x = np.concatenate([fluid, wall])
    kind = np.concatenate([np.zeros(len(fluid), np.int8), np.ones(len(wall), np.int8)])
    h = np.concatenate([h_f, np.full(len(wall), H_OVER_DP * dpf)])
    m = np.concatenate([rho0 * dp_f ** 2, np.full(len(wall), rho0 * dpf ** 2)])
    v = np.zeros_like(x)
    v[kind == 0, 0] = U
    nu = U * D / Re
    return _case("cylinder2d", 2, (0, 0, 0), (box[0], box[1], 1.0), (1, 1, 0), rho0, c0, rho0 * nu, U, x, v,
                 h, m, kind=kind, dp=dpc, dp_min=dpf, Re=Re, U=U, nu=nu, seed=seed,
                 n_fluid=len(fluid), n_wall=len(wall))


def lattice_block(dim: int, n: int, dp: float = 1.0, periodic: bool = True, jitter_dp: float = 0.0,
                  seed: int = SEED, rho0: float = 1.0, c0: float = 10.0, eta: float = 0.0,
                  h_over_dp: float = H_OVER_DP):
    """A plain n^dim periodic lattice block (spacing dp, optional jitter), at
    rest: the building block of the oracle's invariance tests."""
    counts = (n,) * dim
    x = _lattice(counts, dp, (0.0,) * dim)
    ids = np.arange(len(x))
    if jitter_dp:
        x += jitter(ids, dim, jitter_dp * dp, seed)
    L = (n * dp,) * dim + (1.0,) * (3 - dim)
    per = (int(periodic),) * dim + (0,) * (3 - dim)
    return _case("lattice%dd" % dim, dim, (0, 0, 0), L, per, rho0, c0, eta, 1.0, x, np.zeros_like(x),
                 h_over_dp * dp, rho0 * dp ** dim, dp=dp)
