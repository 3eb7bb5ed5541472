"""FP64 CPU oracle of the transport-velocity WCSPH kick-drift-kick step.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow reference the CUDA
library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the library itself never
does, and the two share no code.

The arithmetic lives in ``sph_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off``); this module only builds it with gcc, loads it with
ctypes and marshals numpy arrays.  Vectors are (N, 3) float64 arrays, with a
zero third column in 2-D.

Functions and the passages they follow (paper sections / equations):

* ``kernel_W``, ``kernel_dW`` -- Wendland C2 kernel, support 2h (Sec. 4).
* ``lattice_sum`` -- the reference sum of Eq. 8 on a perfect lattice.
* ``neighbours`` -- all j with |x_i - x_j| < 2 h_ij (brute force or cells).
* ``density`` -- Eq. 8 with Eq. 2.
* ``forces`` -- Eq. 3 (row 2), 5, 6, 7 and Eq. 14-16 (plus the free-stream
  forcing of ``fringe_rate`` when it is switched on).
* ``fringe_rate`` -- the fringe-region forcing rate (Nordstrom et al. 1999),
  standing in for the free-stream boundary Sec. 4.4 cites without giving it.
* ``wall_force`` -- the force of the fluid on the walls (Eq. 18's F).
* ``time_step`` -- Eq. 9-11.
* ``step`` -- one kick-drift-kick step (Sec. 1, Sec. 3).
* ``viscous``, ``pressure``, ``continuity`` -- Eq. 7, Eq. 3 (row 2) with
  Eq. 5-6, and Eq. 3 (row 1) with U* of Eq. 5 (row 1), each alone.
* ``advection_step``, ``acoustic_step`` -- Eq. 9-10 and Eq. 11.
* ``dual_step`` -- one advection step of the dual-criteria scheme (Sec. 2.4,
  the correction once per advection step as in Sec. 3, Eq. 12-13 for the
  background-pressure form).

Pins (tests/test_oracle_*.py): kernel normalisation by quadrature and its
derivative by finite differences; lattice partition of unity and zero
residual; linear pressure and quadratic velocity fields (gradient and
Laplacian consistency, which fix the factors and signs of Eq. 3 and Eq. 7);
pairwise momentum and central-force angular momentum conservation; Galilean
and translation invariance; Riemann limiter scaling; limiter values from
Eq. 15; the Taylor-Green kinetic-energy decay exp(-16 pi^2 nu t).  The wall
branch and the variable-resolution pair smoothing length are PARITY UNPINNED
(the paper states neither).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIBPATH = os.path.join(_BUILD, "libsph_oracle.so")
_lock = threading.Lock()
_lib = None

TV_NONE, TV_LIMITED, TV_UNLIMITED, TV_BACKGROUND = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP if available).  Returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIBPATH) and os.path.getmtime(_LIBPATH) >= os.path.getmtime(_SRC):
        return _LIBPATH
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
    tmp = _LIBPATH + ".tmp%d" % os.getpid()
    try:
        subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [_SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIBPATH)
    return _LIBPATH


class Params(ctypes.Structure):
    """Mirror of ``orc_params`` in sph_oracle.c."""

    _fields_ = [
        ("dim", ctypes.c_int32),
        ("periodic", ctypes.c_int32 * 3),
        ("lo", ctypes.c_double * 3),
        ("L", ctypes.c_double * 3),
        ("rho0", ctypes.c_double),
        ("c", ctypes.c_double),
        ("eta", ctypes.c_double),
        ("g", ctypes.c_double * 3),
        ("h_min", ctypes.c_double),
        ("riemann_eta", ctypes.c_double),
        ("tv_mode", ctypes.c_int32),
        ("tv_h_per_particle", ctypes.c_int32),
        ("tv_xi", ctypes.c_double),
        ("tv_C", ctypes.c_double),
        ("tv_thresh", ctypes.c_double),
        ("h_pair_max", ctypes.c_int32),
        ("pad0", ctypes.c_int32),
        ("cfl_ad", ctypes.c_double),
        ("cfl_ac", ctypes.c_double),
        ("u_ref", ctypes.c_double),
        ("dt_tv", ctypes.c_double),
        ("tv_p0", ctypes.c_double),
        ("fs_lambda", ctypes.c_double),
        ("fs_u", ctypes.c_double * 3),
        ("fs_x", ctypes.c_double * 4),
    ]


def make_params(dim, lo, L, periodic, rho0, c, eta, h_min, g=(0.0, 0.0, 0.0), u_ref=0.0,
                tv_mode=TV_LIMITED, tv_h_per_particle=False, h_pair_max=False,
                riemann_eta=3.0, tv_xi=-0.2, tv_C=1.0e3, tv_thresh=5.0e-4,
                cfl_ad=0.25, cfl_ac=0.6, fringe=None) -> Params:
    """Oracle parameters; defaults are the paper's constants (Eq. 6, 9-11, 15, 16).
    fringe = (lambda_max, (Ux, Uy, Uz), (x_start, x_end, rise, fall)) switches
    on the free-stream forcing of ``fringe_rate``."""
    P = Params()
    P.dim = int(dim)
    for d in range(3):
        P.periodic[d] = int(bool(periodic[d])) if d < len(periodic) else 0
        P.lo[d] = float(lo[d]) if d < len(lo) else 0.0
        P.L[d] = float(L[d]) if d < len(L) else 1.0
        P.g[d] = float(g[d]) if d < len(g) else 0.0
    P.rho0, P.c, P.eta, P.h_min = float(rho0), float(c), float(eta), float(h_min)
    P.riemann_eta = float(riemann_eta)
    P.tv_mode, P.tv_h_per_particle = int(tv_mode), int(bool(tv_h_per_particle))
    P.tv_xi, P.tv_C, P.tv_thresh = float(tv_xi), float(tv_C), float(tv_thresh)
    P.h_pair_max = int(bool(h_pair_max))
    P.cfl_ad, P.cfl_ac, P.u_ref = float(cfl_ad), float(cfl_ac), float(u_ref)
    if fringe is not None:
        lam, u, xs = fringe
        P.fs_lambda = float(lam)
        for d in range(3):
            P.fs_u[d] = float(u[d])
        for k in range(4):
            P.fs_x[k] = float(xs[k])
    return P


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int64)
_bp = ctypes.POINTER(ctypes.c_int8)
_pp = ctypes.POINTER(Params)
_i64 = ctypes.c_int64


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            sig = {
                "orc_set_threads": (None, [ctypes.c_int]),
                "orc_get_threads": (ctypes.c_int, []),
                "orc_kernel_W": (ctypes.c_double, [ctypes.c_double, ctypes.c_double, ctypes.c_int]),
                "orc_kernel_dW": (ctypes.c_double, [ctypes.c_double, ctypes.c_double, ctypes.c_int]),
                "orc_lattice_sum": (ctypes.c_double, [ctypes.c_int, ctypes.c_double]),
                "orc_pair_h": (ctypes.c_double, [_pp, ctypes.c_double, ctypes.c_double]),
                "orc_eos": (ctypes.c_double, [_pp, ctypes.c_double]),
                "orc_riemann_beta": (ctypes.c_double, [_pp, ctypes.c_double, ctypes.c_double]),
                "orc_riemann_pstar": (ctypes.c_double, [_pp] + [ctypes.c_double] * 5),
                "orc_tv_limiter": (ctypes.c_double, [_pp, ctypes.c_double]),
                "orc_neighbours": (_i64, [_pp, _i64, _dp, _dp, ctypes.c_int, _ip, _ip]),
                "orc_density": (None, [_pp, _i64, _dp, _dp, _bp, _dp, _ip, _ip, _dp, _dp]),
                "orc_forces": (None, [_pp, _i64, _dp, _dp, _dp, _dp, _bp, _dp, _dp, _ip, _ip,
                                      _dp, _dp, _dp, _dp]),
                "orc_kick": (None, [_pp, _i64, ctypes.c_double, _dp, _dp, _bp]),
                "orc_drift": (None, [_pp, _i64, ctypes.c_double, _dp, _dp, _dp, _bp]),
                "orc_time_step": (ctypes.c_double, [_pp, _i64, _dp, _bp]),
                "orc_diagnostics": (None, [_pp, _i64, _dp, _dp, _bp, _dp, _dp, ctypes.c_double, _dp]),
                "orc_force_pass": (ctypes.c_int, [_pp, _i64, _dp, _dp, _dp, _dp, _bp, _dp, _dp,
                                                  ctypes.c_int, _dp, _dp, _dp, _dp, _dp]),
                "orc_step": (ctypes.c_int, [_pp, _i64, _dp, _dp, _dp, _dp, _dp, _dp, _bp, _dp, _dp,
                                            ctypes.c_double, ctypes.c_int, _dp, _dp, _dp]),
                "orc_kernel_d2W": (ctypes.c_double, [ctypes.c_double, ctypes.c_double, ctypes.c_int]),
                "orc_riemann_dbeta": (ctypes.c_double, [_pp, ctypes.c_double]),
                "orc_tv_dlimiter": (ctypes.c_double, [_pp, ctypes.c_double]),
                "orc_step_adjoint": (ctypes.c_int, [_pp, _i64, _dp, _dp, _dp, _dp, _dp, _dp, _bp, _dp, _dp,
                                                    ctypes.c_double, ctypes.c_int, _dp, _dp, _dp, _dp, _dp]),
                "orc_force_pass_adjoint": (ctypes.c_int, [_pp, _i64, _dp, _dp, _dp, _dp, _bp, _dp, _dp,
                                                          ctypes.c_int, _dp, _dp, _dp, _dp, _dp]),
                "orc_viscous": (None, [_pp, _i64, _dp, _dp, _dp, _dp, _bp, _dp, _dp, _ip, _ip, _dp]),
                "orc_pressure": (None, [_pp, _i64, _dp, _dp, _dp, _dp, _bp, _dp, _dp, _ip, _ip, _dp]),
                "orc_continuity": (None, [_pp, _i64, _dp, _dp, _dp, _dp, _bp, _dp, _dp, _ip, _ip, _dp]),
                "orc_riemann_ustar": (ctypes.c_double, [_pp] + [ctypes.c_double] * 5),
                "orc_fringe": (ctypes.c_double, [_pp, ctypes.c_double]),
                "orc_wall_force": (None, [_pp, _i64, _dp, _dp, _dp, _dp, _bp, _dp, _dp, _ip, _ip, _dp]),
                "orc_advection_step": (ctypes.c_double, [_pp, _i64, _dp, _bp, _dp]),
                "orc_acoustic_step": (ctypes.c_double, [_pp, _i64, _dp, _bp]),
                "orc_dual_step": (_i64, [_pp, _i64, _dp, _dp, _dp, _dp, _dp, _dp, _bp, _dp, _dp, ctypes.c_int,
                                         _dp, _dp, _dp, _dp, _dp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def _d(a):
    return a.ctypes.data_as(_dp)


def _vec(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape == (n, 2):
        a = np.concatenate([a, np.zeros((n, 1))], axis=1)
    assert a.shape == (n, 3), a.shape
    return np.ascontiguousarray(a)


def _sca(a, n, dtype=np.float64):
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=dtype), (n,)), dtype=dtype)
    return a


def kernel_W(r, h, dim):
    return lib().orc_kernel_W(float(r), float(h), int(dim))


def kernel_dW(r, h, dim):
    return lib().orc_kernel_dW(float(r), float(h), int(dim))


def lattice_sum(dim, h_over_dp=1.3):
    """sum_k W(|k|, h_over_dp) over the unit integer lattice (sigma0 * dp^D)."""
    return lib().orc_lattice_sum(int(dim), float(h_over_dp))


def pair_h(P, hi, hj):
    return lib().orc_pair_h(ctypes.byref(P), float(hi), float(hj))


def eos(P, rho):
    return lib().orc_eos(ctypes.byref(P), float(rho))


def riemann_beta(P, ul, ur):
    return lib().orc_riemann_beta(ctypes.byref(P), float(ul), float(ur))


def riemann_pstar(P, pl, pr, rhobar, ul, ur):
    return lib().orc_riemann_pstar(ctypes.byref(P), float(pl), float(pr), float(rhobar), float(ul), float(ur))


def tv_limiter(P, s):
    return lib().orc_tv_limiter(ctypes.byref(P), float(s))


def neighbours(P, x, h, mode="cells"):
    """CSR neighbour lists (self included, ascending j): returns (start, idx)."""
    n = len(x)
    x = _vec(x, n)
    h = _sca(h, n)
    m = {"brute": 0, "cells": 1}[mode]
    start = np.zeros(n + 1, dtype=np.int64)
    tot = lib().orc_neighbours(ctypes.byref(P), n, _d(x), _d(h), m, start.ctypes.data_as(_ip), None)
    idx = np.zeros(max(int(tot), 1), dtype=np.int64)
    lib().orc_neighbours(ctypes.byref(P), n, _d(x), _d(h), m, start.ctypes.data_as(_ip), idx.ctypes.data_as(_ip))
    return start, idx[: int(tot)]


def density(P, x, h, kind, sigma0, nbrs):
    """Eq. 8: returns (rho, sigma)."""
    n = len(x)
    x, h, s0 = _vec(x, n), _sca(h, n), _sca(sigma0, n)
    kind = _sca(kind, n, np.int8)
    start, idx = nbrs
    idx = np.ascontiguousarray(idx, dtype=np.int64) if len(idx) else np.zeros(1, np.int64)
    rho, sigma = np.zeros(n), np.zeros(n)
    lib().orc_density(ctypes.byref(P), n, _d(x), _d(h), kind.ctypes.data_as(_bp), _d(s0),
                      start.ctypes.data_as(_ip), idx.ctypes.data_as(_ip), _d(rho), _d(sigma))
    return rho, sigma


def forces(P, x, v, h, m, kind, vw, rho, nbrs):
    """Eq. 3, 5-7, 14-16: returns dict a, R, chi, dr."""
    n = len(x)
    x, v, vw = _vec(x, n), _vec(v, n), _vec(vw, n)
    h, m, rho = _sca(h, n), _sca(m, n), _sca(rho, n)
    kind = _sca(kind, n, np.int8)
    start, idx = nbrs
    idx = np.ascontiguousarray(idx, dtype=np.int64) if len(idx) else np.zeros(1, np.int64)
    a, R, dr = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3))
    chi = np.zeros(n)
    lib().orc_forces(ctypes.byref(P), n, _d(x), _d(v), _d(h), _d(m), kind.ctypes.data_as(_bp), _d(vw), _d(rho),
                     start.ctypes.data_as(_ip), idx.ctypes.data_as(_ip), _d(a), _d(R), _d(chi), _d(dr))
    return {"a": a, "R": R, "chi": chi, "dr": dr}


def fringe_rate(P, x):
    """lambda(x) of the free-stream forcing lambda(x) (U_inf - v) (fringe
    region along axis 0; 0 when P.fs_lambda is 0)."""
    return lib().orc_fringe(ctypes.byref(P), float(x))


def wall_force(P, x, v, h, m, kind, vw, rho, nbrs):
    """Force of the fluid on the wall particles (the body of Eq. 18): minus
    the sum over fluid i of m_i times its wall neighbours' pressure and
    viscous terms.  Returns a 3-vector."""
    n = len(x)
    x, v, vw = _vec(x, n), _vec(v, n), _vec(vw, n)
    h, m, rho = _sca(h, n), _sca(m, n), _sca(rho, n)
    kind = _sca(kind, n, np.int8)
    start, idx = nbrs
    idx = np.ascontiguousarray(idx, dtype=np.int64) if len(idx) else np.zeros(1, np.int64)
    F = np.zeros(3)
    lib().orc_wall_force(ctypes.byref(P), n, _d(x), _d(v), _d(h), _d(m), kind.ctypes.data_as(_bp), _d(vw),
                         _d(rho), start.ctypes.data_as(_ip), idx.ctypes.data_as(_ip), _d(F))
    return F


def time_step(P, v, kind):
    """Eq. 9-11 with h = h_min."""
    n = len(v)
    v = _vec(v, n)
    kind = _sca(kind, n, np.int8)
    return lib().orc_time_step(ctypes.byref(P), n, _d(v), kind.ctypes.data_as(_bp))


def diagnostics(P, v, m, kind, dr, chi, dt):
    """mass, momentum[3], KE, max|v|, max overcorrection ratio, count chi>0."""
    n = len(v)
    v, dr = _vec(v, n), _vec(dr, n)
    m, chi = _sca(m, n), _sca(chi, n)
    kind = _sca(kind, n, np.int8)
    out = np.zeros(8)
    lib().orc_diagnostics(ctypes.byref(P), n, _d(v), _d(m), kind.ctypes.data_as(_bp), _d(dr), _d(chi),
                          float(dt), _d(out))
    return {"mass": out[0], "momentum": out[1:4].copy(), "ke": out[4], "vmax": out[5],
            "overcorrection": out[6], "n_chi": int(out[7])}


def _case_arrays(case, n):
    h = _sca(case["h"], n)
    m = _sca(case["m"], n)
    kind = _sca(case.get("kind", 0), n, np.int8)
    vw = _vec(case.get("vw", np.zeros((n, 3))), n)
    return h, m, kind, vw


def force_pass(P, case, x, v, sigma0, mode="cells"):
    """Neighbours + density + forces on (x, v): returns dict rho, a, R, chi, dr."""
    n = len(x)
    x, v = _vec(x, n), _vec(v, n)
    h, m, kind, vw = _case_arrays(case, n)
    s0 = _sca(sigma0, n)
    rho, chi = np.zeros(n), np.zeros(n)
    a, R, dr = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3))
    rc = lib().orc_force_pass(ctypes.byref(P), n, _d(x), _d(v), _d(h), _d(m), kind.ctypes.data_as(_bp), _d(vw),
                              _d(s0), {"brute": 0, "cells": 1}[mode], _d(rho), _d(a), _d(R), _d(chi), _d(dr))
    if rc:
        raise MemoryError("oracle force pass failed")
    return {"rho": rho, "a": a, "R": R, "chi": chi, "dr": dr}


def step(P, case, state, sigma0, dt, mode="cells"):
    """One kick-drift-kick step.  ``state`` holds x, v, a, dr ((N,3) float64);
    returns a new dict with x, v, a, dr, rho, R, chi (inputs untouched)."""
    n = len(state["x"])
    x, v = _vec(state["x"], n).copy(), _vec(state["v"], n).copy()
    a, dr = _vec(state["a"], n).copy(), _vec(state["dr"], n).copy()
    h, m, kind, vw = _case_arrays(case, n)
    s0 = _sca(sigma0, n)
    rho, chi, R = np.zeros(n), np.zeros(n), np.zeros((n, 3))
    rc = lib().orc_step(ctypes.byref(P), n, _d(x), _d(v), _d(a), _d(dr), _d(h), _d(m), kind.ctypes.data_as(_bp),
                        _d(vw), _d(s0), float(dt), {"brute": 0, "cells": 1}[mode], _d(rho), _d(R), _d(chi))
    if rc:
        raise MemoryError("oracle step failed")
    return {"x": x, "v": v, "a": a, "dr": dr, "rho": rho, "R": R, "chi": chi}


def kick(P, v, a, kind, hdt):
    """v += hdt a for fluid particles (returns a new array)."""
    n = len(v)
    v = _vec(v, n).copy()
    a = _vec(a, n)
    kind = _sca(kind, n, np.int8)
    lib().orc_kick(ctypes.byref(P), n, float(hdt), _d(v), _d(a), kind.ctypes.data_as(_bp))
    return v


def drift(P, x, v, dr, kind, dt):
    """x += dt v + dr for fluid particles, periodic wrap (returns a new array)."""
    n = len(x)
    x = _vec(x, n).copy()
    v, dr = _vec(v, n), _vec(dr, n)
    kind = _sca(kind, n, np.int8)
    lib().orc_drift(ctypes.byref(P), n, float(dt), _d(x), _d(v), _d(dr), kind.ctypes.data_as(_bp))
    return x


def reverse_segments(start, idx):
    """The CSR neighbour lists with every particle's list reversed."""
    counts = np.diff(start)
    seg = np.repeat(np.arange(len(counts)), counts)
    k = np.arange(len(idx))
    return np.ascontiguousarray(idx[start[seg] + start[seg + 1] - 1 - k])


def step_reversed_sums(P, case, state, sigma0, dt):
    """The same kick-drift-kick step as ``step`` with every neighbour sum taken
    in descending instead of ascending j.  The two results differ only by
    floating-point summation order: their difference measures the rounding
    floor of the method's FP64 arithmetic on this state."""
    n = len(state["x"])
    h, m, kind, vw = _case_arrays(case, n)
    hdt = 0.5 * dt
    saved_dt_tv = P.dt_tv
    P.dt_tv = dt
    v = kick(P, state["v"], state["a"], kind, hdt)
    x = drift(P, state["x"], v, state["dr"], kind, dt)
    start, idx = neighbours(P, x, h)
    nb = (start, reverse_segments(start, idx))
    rho, _ = density(P, x, h, kind, sigma0, nb)
    f = forces(P, x, v, h, m, kind, vw, rho, nb)
    v = kick(P, v, f["a"], kind, hdt)
    P.dt_tv = saved_dt_tv
    return {"x": x, "v": v, "a": f["a"], "dr": f["dr"], "rho": rho, "R": f["R"], "chi": f["chi"]}


def kernel_d2W(r, h, dim):
    return lib().orc_kernel_d2W(float(r), float(h), int(dim))


def step_adjoint(P, case, state, sigma0, dt, cot, mode="cells"):
    """Reverse of ``step`` (neighbour lists and dt frozen).  ``state`` is the
    step's input (x, v, a, dr); ``cot`` holds the cotangents of its outputs
    (x, v, a, dr).  Returns (cotangents of the inputs, d/d eta)."""
    n = len(state["x"])
    x, v = _vec(state["x"], n), _vec(state["v"], n)
    a, dr = _vec(state["a"], n), _vec(state["dr"], n)
    h, m, kind, vw = _case_arrays(case, n)
    s0 = _sca(sigma0, n)
    xb, vb = _vec(cot["x"], n).copy(), _vec(cot["v"], n).copy()
    ab, drb = _vec(cot["a"], n).copy(), _vec(cot["dr"], n).copy()
    eb = ctypes.c_double(0.0)
    rc = lib().orc_step_adjoint(ctypes.byref(P), n, _d(x), _d(v), _d(a), _d(dr), _d(h), _d(m),
                                kind.ctypes.data_as(_bp), _d(vw), _d(s0), float(dt), {"brute": 0, "cells": 1}[mode],
                                _d(xb), _d(vb), _d(ab), _d(drb), ctypes.byref(eb))
    if rc:
        raise MemoryError("oracle step adjoint failed")
    return {"x": xb, "v": vb, "a": ab, "dr": drb}, eb.value


def force_pass_adjoint(P, case, x, v, sigma0, abar, drbar, mode="cells"):
    """Reverse of ``force_pass``: cotangents of (x, v) and d/d eta from those
    of (a, dr)."""
    n = len(x)
    x, v = _vec(x, n), _vec(v, n)
    h, m, kind, vw = _case_arrays(case, n)
    s0 = _sca(sigma0, n)
    A, D = _vec(abar, n), _vec(drbar, n)
    xb, vb = np.zeros((n, 3)), np.zeros((n, 3))
    eb = ctypes.c_double(0.0)
    rc = lib().orc_force_pass_adjoint(ctypes.byref(P), n, _d(x), _d(v), _d(h), _d(m), kind.ctypes.data_as(_bp),
                                      _d(vw), _d(s0), {"brute": 0, "cells": 1}[mode], _d(A), _d(D), _d(xb), _d(vb),
                                      ctypes.byref(eb))
    if rc:
        raise MemoryError("oracle force-pass adjoint failed")
    return xb, vb, eb.value


def rollout(P, case, x0, v0, sigma0, dt, nsteps, mode="cells"):
    """Initial force pass on (x0, v0), then ``nsteps`` steps: the states
    [s_0, ..., s_T] (each a dict x, v, a, dr, ...)."""
    fp = force_pass(P, case, x0, v0, sigma0, mode)
    st = {"x": _vec(x0, len(x0)).copy(), "v": _vec(v0, len(v0)).copy(), "a": fp["a"], "dr": fp["dr"],
          "rho": fp["rho"]}
    out = [st]
    for _ in range(nsteps):
        st = step(P, case, st, sigma0, dt, mode)
        out.append(st)
    return out


def rollout_adjoint(P, case, states, sigma0, dt, cot_T, mode="cells"):
    """Gradients of a loss with cotangents ``cot_T`` (x, v, a, dr of the last
    state) back to (x0, v0) and eta, through every step and the initial
    force pass."""
    cot = {k: np.array(v, dtype=np.float64) for k, v in cot_T.items()}
    eta_bar = 0.0
    for k in range(len(states) - 1, 0, -1):
        cot, eb = step_adjoint(P, case, states[k - 1], sigma0, dt, cot, mode)
        eta_bar += eb
    xb, vb, eb = force_pass_adjoint(P, case, states[0]["x"], states[0]["v"], sigma0, cot["a"], cot["dr"], mode)
    return cot["x"] + xb, cot["v"] + vb, eta_bar + eb


def sigma0_for(case, dim):
    """Per-particle reference sum of Eq. 8: the perfect-lattice sum at the
    particle's own spacing dp = (m / rho0)^(1/D) and smoothing length h."""
    h = np.asarray(case["h"], dtype=np.float64)
    m = np.asarray(case["m"], dtype=np.float64)
    dp = (m / case["rho0"]) ** (1.0 / dim)
    out = np.empty(len(h))
    pairs, inv = np.unique(np.stack([h, dp], axis=1), axis=0, return_inverse=True)
    vals = np.array([lattice_sum(dim, hh / dd) / dd ** dim for hh, dd in pairs])
    out[:] = vals[np.ravel(inv)]
    return out


# ----------------------------------------------------- dual-criteria stepping

def _pair_fn(name, P, x, v, h, m, kind, vw, rho, nbrs, width):
    n = len(x)
    x, v, vw = _vec(x, n), _vec(v, n), _vec(vw, n)
    h, m, rho = _sca(h, n), _sca(m, n), _sca(rho, n)
    kind = _sca(kind, n, np.int8)
    start, idx = nbrs
    idx = np.ascontiguousarray(idx, dtype=np.int64) if len(idx) else np.zeros(1, np.int64)
    out = np.zeros((n, 3)) if width == 3 else np.zeros(n)
    getattr(lib(), name)(ctypes.byref(P), n, _d(x), _d(v), _d(h), _d(m), kind.ctypes.data_as(_bp), _d(vw), _d(rho),
                         start.ctypes.data_as(_ip), idx.ctypes.data_as(_ip), _d(out))
    return out


def viscous(P, x, v, h, m, kind, vw, rho, nbrs):
    """Eq. 7 alone: the viscous acceleration (N, 3)."""
    return _pair_fn("orc_viscous", P, x, v, h, m, kind, vw, rho, nbrs, 3)


def pressure(P, x, v, h, m, kind, vw, rho, nbrs):
    """Eq. 3 (row 2) with Eq. 5-6 alone: the pressure acceleration (N, 3)."""
    return _pair_fn("orc_pressure", P, x, v, h, m, kind, vw, rho, nbrs, 3)


def continuity(P, x, v, h, m, kind, vw, rho, nbrs):
    """Eq. 3 (row 1) with U* of Eq. 5 (row 1): d rho / dt (N,)."""
    return _pair_fn("orc_continuity", P, x, v, h, m, kind, vw, rho, nbrs, 1)


def riemann_ustar(P, pl, pr, rhobar, ul, ur):
    return lib().orc_riemann_ustar(ctypes.byref(P), pl, pr, rhobar, ul, ur)


def advection_step(P, v, kind):
    """Eq. 9-10 with h = h_min: returns (Dt_ad, |v|_ad)."""
    n = len(v)
    v = _vec(v, n)
    kind = _sca(kind, n, np.int8)
    vad = ctypes.c_double(0.0)
    dt = lib().orc_advection_step(ctypes.byref(P), n, _d(v), kind.ctypes.data_as(_bp), ctypes.byref(vad))
    return dt, vad.value


def acoustic_step(P, v, kind):
    """Eq. 11 with h = h_min."""
    n = len(v)
    v = _vec(v, n)
    kind = _sca(kind, n, np.int8)
    return lib().orc_acoustic_step(ctypes.byref(P), n, _d(v), kind.ctypes.data_as(_bp))


def dual_step(P, case, state, sigma0, mode="cells"):
    """One advection step of the dual-criteria scheme.  ``state`` holds x, v
    ((N, 3) float64) and drho ((N,), zero at the start of a run); returns a
    new dict with x, v, rho, drho, a (last substep), dr, R, chi, Dt and the
    number of acoustic substeps (inputs untouched)."""
    n = len(state["x"])
    x, v = _vec(state["x"], n).copy(), _vec(state["v"], n).copy()
    drho = _sca(state.get("drho", 0.0), n).copy()
    h, m, kind, vw = _case_arrays(case, n)
    s0 = _sca(sigma0, n)
    rho, chi = np.zeros(n), np.zeros(n)
    a, dr, R = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3))
    Dt = ctypes.c_double(0.0)
    k = lib().orc_dual_step(ctypes.byref(P), n, _d(x), _d(v), _d(rho), _d(drho), _d(h), _d(m),
                            kind.ctypes.data_as(_bp), _d(vw), _d(s0), {"brute": 0, "cells": 1}[mode], _d(a), _d(dr),
                            _d(R), _d(chi), ctypes.byref(Dt))
    if k < 0:
        raise MemoryError("oracle dual step failed")
    return {"x": x, "v": v, "rho": rho, "drho": drho, "a": a, "dr": dr, "R": R, "chi": chi, "Dt": Dt.value,
            "substeps": int(k)}
