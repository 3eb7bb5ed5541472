"""paper_2411_13992_gb300 -- GB300-native transport-velocity WCSPH step.

Thin Python binding of libsphtv (C ABI in include/sphtv.h).  Each ``sph_*``
function here marshals arguments for the C function of the same name and
nothing else: every step of the method runs in the library's CUDA kernels.
PyTorch only provides device memory (the workspace) and the stream.

The library is loaded lazily on first use; if it is missing or cannot be
loaded the call raises -- there is no CPU fallback.

Method (arXiv 2411.13992, Wang, Haidn & Hu): weakly-compressible SPH with a
Riemann-based pressure force (Eq. 3, 5-6), viscous force (Eq. 7), summation
density (Eq. 8) and the h^2-scaled, limited transport-velocity correction
(Eq. 14-16), advanced by kick-drift-kick steps of size min(dt_ad, dt_ac)
(Eq. 9-11).
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

from . import _build

__all__ = [
    "SphParams", "SphDiag", "SphError", "load", "exported_symbols", "declared_symbols",
    "sph_default_params", "sph_query_workspace", "sph_create", "sph_set_state", "sph_build_cells", "sph_step",
    "sph_set_dt", "sph_set_eta", "sph_get_state", "sph_get_diag", "sph_sync", "sph_destroy", "sph_status_str",
    "sph_launch_count", "sph_profile_begin", "sph_profile_end", "sph_kernel_class_name", "KERNEL_CLASSES", "sph_fma_peak",
    "sph_density_noalloc", "NOALLOC_MAX_PARTICLES", "sph_step_adjoint", "sph_force_pass_adjoint", "SphCkpt",
    "sph_save_ckpt",
    "params_from_case", "Simulation", "Rollout",
    "TV_OFF", "TV_LIMITED", "TV_UNLIMITED", "TV_BACKGROUND", "TVH_MIN", "TVH_PARTICLE", "HPAIR_MEAN", "HPAIR_MAX",
    "INT_KDK", "INT_DUAL", "sph_set_density_rate", "sph_get_density_rate",
]

TV_OFF, TV_LIMITED, TV_UNLIMITED, TV_BACKGROUND = 0, 1, 2, 3
INT_KDK, INT_DUAL = 0, 1
TVH_MIN, TVH_PARTICLE = 0, 1
HPAIR_MEAN, HPAIR_MAX = 0, 1

STATUS_NAMES = {0: "SPH_OK", 1: "SPH_ERR_ARG", 2: "SPH_ERR_CUDA", 3: "SPH_ERR_WORKSPACE", 4: "SPH_ERR_OVERFLOW",
                5: "SPH_ERR_NAN", 6: "SPH_ERR_DOMAIN", 7: "SPH_ERR_STATE", 8: "SPH_ERR_INPUT"}

HEADER = os.path.join(_build.INCLUDE, "sphtv.h")


class SphParams(ctypes.Structure):
    """Mirror of ``sph_params``."""

    _fields_ = [
        ("dim", ctypes.c_int32), ("precision", ctypes.c_int32), ("periodic", ctypes.c_int32 * 3),
        ("tv_mode", ctypes.c_int32),
        ("lo", ctypes.c_double * 3), ("L", ctypes.c_double * 3),
        ("rho0", ctypes.c_double), ("c0", ctypes.c_double), ("eta", ctypes.c_double), ("g", ctypes.c_double * 3),
        ("h_min", ctypes.c_double), ("h_max", ctypes.c_double), ("riemann_eta", ctypes.c_double),
        ("tv_xi", ctypes.c_double), ("tv_C", ctypes.c_double), ("tv_thresh", ctypes.c_double),
        ("cfl_ad", ctypes.c_double), ("cfl_ac", ctypes.c_double), ("u_ref", ctypes.c_double),
        ("fixed_dt", ctypes.c_double),
        ("tv_h", ctypes.c_int32), ("h_pair", ctypes.c_int32), ("kahan", ctypes.c_int32),
        ("adjoint_steps", ctypes.c_int32), ("integrator", ctypes.c_int32), ("graphs", ctypes.c_int32),
        ("pair_tiles", ctypes.c_int32), ("body_force", ctypes.c_int32),
        ("fringe_lambda", ctypes.c_double), ("fringe_u", ctypes.c_double * 3), ("fringe_x", ctypes.c_double * 4),
        ("x_subcells", ctypes.c_int32),
    ]


class SphDiag(ctypes.Structure):
    """Mirror of ``sph_diag``."""

    _fields_ = [
        ("mass", ctypes.c_double), ("momentum", ctypes.c_double * 3), ("kinetic", ctypes.c_double),
        ("vmax", ctypes.c_double), ("vt_max", ctypes.c_double), ("dr_max", ctypes.c_double),
        ("n_chi", ctypes.c_double), ("dt", ctypes.c_double), ("dt_next", ctypes.c_double),
        ("steps", ctypes.c_double), ("substeps", ctypes.c_double), ("body_force", ctypes.c_double * 3),
        ("body_impulse", ctypes.c_double * 3), ("time", ctypes.c_double),
    ]

    def as_dict(self):
        return {"mass": self.mass, "momentum": np.array(self.momentum[:]), "ke": self.kinetic, "vmax": self.vmax,
                "vt_max": self.vt_max, "dr_max": self.dr_max, "n_chi": int(self.n_chi), "dt": self.dt,
                "dt_next": self.dt_next, "steps": int(self.steps), "substeps": int(self.substeps),
                "body_force": np.array(self.body_force[:]), "body_impulse": np.array(self.body_impulse[:]),
                "time": self.time}


class SphCkpt(ctypes.Structure):
    """Mirror of ``sph_ckpt``."""

    _fields_ = [("x", ctypes.c_void_p), ("v", ctypes.c_void_p), ("a", ctypes.c_void_p), ("dr", ctypes.c_void_p),
                ("dt_next", ctypes.c_double), ("steps", ctypes.c_double)]


class SphError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s failed: %s (%s)" % (where, STATUS_NAMES.get(status, status), _status_str(status)))


_lock = threading.Lock()
_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libsphtv.so (building it with nvcc first if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.lib_path()
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError("libsphtv.so is not built (%s)" % path)
            _build.build()
        L = ctypes.CDLL(path)
        pP = ctypes.POINTER(SphParams)
        sig = {
            "sph_default_params": (_i32, [pP]),
            "sph_query_workspace": (_i32, [pP, _i64, ctypes.POINTER(ctypes.c_size_t)]),
            "sph_create": (_i32, [pP, _i64, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(_vp)]),
            "sph_set_state": (_i32, [_vp] + [_vp] * 9),
            "sph_build_cells": (_i32, [_vp]),
            "sph_step": (_i32, [_vp, _i32]),
            "sph_set_dt": (_i32, [_vp, ctypes.c_double]),
            "sph_set_eta": (_i32, [_vp, ctypes.c_double]),
            "sph_get_state": (_i32, [_vp] + [_vp] * 5),
            "sph_get_diag": (_i32, [_vp, ctypes.POINTER(SphDiag)]),
            "sph_save_ckpt": (_i32, [_vp, ctypes.POINTER(SphCkpt)]),
            "sph_sync": (_i32, [_vp]),
            "sph_destroy": (None, [_vp]),
            "sph_status_str": (ctypes.c_char_p, [_i32]),
            "sph_launch_count": (_i64, [_vp]),
            "sph_profile_begin": (_i32, [_vp, _i32]),
            "sph_profile_end": (_i32, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64)]),
            "sph_kernel_class_name": (ctypes.c_char_p, [_i32]),
            "sph_density_noalloc": (_i32, [pP, _i64] + [_vp] * 7),
            "sph_step_adjoint": (_i32, [_vp, _vp, _vp, _vp, _vp, _i32, _vp, _vp, _vp, _vp,
                                        ctypes.POINTER(ctypes.c_double)]),
            "sph_force_pass_adjoint": (_i32, [_vp] + [_vp] * 6 + [ctypes.POINTER(ctypes.c_double)]),
            "sph_fma_peak": (_i32, [_i32, _i32, _i32, _vp, _vp, ctypes.POINTER(ctypes.c_double)]),
            "sph_set_density_rate": (_i32, [_vp, _vp]),
            "sph_get_density_rate": (_i32, [_vp, _vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def declared_symbols() -> list:
    """Entry points declared in include/sphtv.h."""
    with open(HEADER) as f:
        text = f.read()
    return re.findall(r"^SPH_API\s+[\w\s\*]+?\b(sph_\w+)\s*\(", text, flags=re.M)


def exported_symbols() -> list:
    lib = load()
    return [s for s in declared_symbols() if hasattr(lib, s)]


def _status_str(status: int) -> str:
    try:
        return load().sph_status_str(int(status)).decode()
    except Exception:  # noqa: BLE001 - only for error messages
        return "?"


def _check(status: int, where: str) -> None:
    if status != 0:
        raise SphError(int(status), where)


# ------------------------------------------------------------------ marshalling

_ASYNC_TEMP = object()   # marker in a keep list: a temporary read after the call returns


def _ptr(a, keep: list, dtype, shape_tail=None):
    """Pointer to a contiguous array of ``dtype`` (numpy or torch), or None."""
    if a is None:
        return None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            tdt = {np.float64: torch.float64, np.int8: torch.int8}[dtype]
            t = a.detach().to(tdt).contiguous()
            if shape_tail == 3 and t.dim() == 2 and t.shape[1] == 2:
                t = torch.nn.functional.pad(t, (0, 1))
            keep.append(t)
            if t.data_ptr() != a.data_ptr() and (t.is_cuda or t.is_pinned()):
                # a converted copy that the library reads asynchronously (in
                # place, or by an asynchronous copy): the caller of the ABI
                # wrapper waits for the stream before it is dropped
                keep.append(_ASYNC_TEMP)
            return t.data_ptr()
    except ImportError:
        pass
    arr = np.ascontiguousarray(a, dtype=dtype)
    if shape_tail == 3 and arr.ndim == 2 and arr.shape[1] == 2:
        arr = np.ascontiguousarray(np.concatenate([arr, np.zeros((len(arr), 1), dtype)], axis=1))
    keep.append(arr)
    return arr.ctypes.data


# ---------------------------------------------------------- ABI-named wrappers

def sph_default_params() -> SphParams:
    p = SphParams()
    _check(load().sph_default_params(ctypes.byref(p)), "sph_default_params")
    return p


def sph_query_workspace(params: SphParams, n: int) -> int:
    b = ctypes.c_size_t(0)
    _check(load().sph_query_workspace(ctypes.byref(params), int(n), ctypes.byref(b)), "sph_query_workspace")
    return int(b.value)


def sph_create(params: SphParams, n: int, workspace_ptr: int, nbytes: int, stream_ptr: int):
    ctx = _vp()
    _check(load().sph_create(ctypes.byref(params), int(n), _vp(workspace_ptr), nbytes, _vp(stream_ptr),
                             ctypes.byref(ctx)), "sph_create")
    return ctx


def sph_set_state(ctx, x, v, a=None, dr=None, h=None, m=None, kind=None, vw=None, sigma0=None) -> None:
    keep = []
    args = [_ptr(x, keep, np.float64, 3), _ptr(v, keep, np.float64, 3), _ptr(a, keep, np.float64, 3),
            _ptr(dr, keep, np.float64, 3), _ptr(h, keep, np.float64), _ptr(m, keep, np.float64),
            _ptr(kind, keep, np.int8), _ptr(vw, keep, np.float64, 3), _ptr(sigma0, keep, np.float64)]
    _check(load().sph_set_state(ctx, *[_vp(p) if p else None for p in args]), "sph_set_state")
    if any(k is _ASYNC_TEMP for k in keep):
        sph_sync(ctx)            # the converted copies must outlive the stream work that reads them


def sph_build_cells(ctx) -> None:
    _check(load().sph_build_cells(ctx), "sph_build_cells")


def sph_step(ctx, nsteps: int = 1) -> None:
    _check(load().sph_step(ctx, int(nsteps)), "sph_step")


def sph_set_dt(ctx, dt: float) -> None:
    _check(load().sph_set_dt(ctx, float(dt)), "sph_set_dt")


def sph_set_eta(ctx, eta: float) -> None:
    _check(load().sph_set_eta(ctx, float(eta)), "sph_set_eta")


def sph_get_state(ctx, x=None, v=None, a=None, dr=None, rho=None) -> None:
    """Write into caller-provided buffers (numpy or torch, contiguous float64)."""
    def p(t):
        if t is None:
            return None
        if hasattr(t, "data_ptr"):
            assert t.is_contiguous()
            return _vp(t.data_ptr())
        assert t.flags["C_CONTIGUOUS"] and t.dtype == np.float64
        return _vp(t.ctypes.data)
    _check(load().sph_get_state(ctx, p(x), p(v), p(a), p(dr), p(rho)), "sph_get_state")


def sph_save_ckpt(ctx, x, v, a, dr):
    """Write a checkpoint into caller-provided [n][3] float64 buffers (numpy or
    torch, contiguous); returns (dt_next, steps)."""
    def p(t):
        if hasattr(t, "data_ptr"):
            assert t.is_contiguous()
            return t.data_ptr()
        assert t.flags["C_CONTIGUOUS"] and t.dtype == np.float64
        return t.ctypes.data
    ck = SphCkpt(p(x), p(v), p(a), p(dr), 0.0, 0.0)
    _check(load().sph_save_ckpt(ctx, ctypes.byref(ck)), "sph_save_ckpt")
    return ck.dt_next, int(ck.steps)


def sph_get_diag(ctx) -> SphDiag:
    d = SphDiag()
    _check(load().sph_get_diag(ctx, ctypes.byref(d)), "sph_get_diag")
    return d


def sph_sync(ctx) -> None:
    _check(load().sph_sync(ctx), "sph_sync (device error)")


def sph_destroy(ctx) -> None:
    load().sph_destroy(ctx)


def sph_status_str(status: int) -> str:
    return _status_str(status)


def sph_launch_count(ctx) -> int:
    return int(load().sph_launch_count(ctx))


KERNEL_CLASSES = 9


def sph_profile_begin(ctx, max_steps: int) -> None:
    _check(load().sph_profile_begin(ctx, int(max_steps)), "sph_profile_begin")


def sph_profile_end(ctx) -> dict:
    """{kernel class name: (summed ms, timed launches)} of the open profile."""
    ms = (ctypes.c_double * KERNEL_CLASSES)()
    cnt = (_i64 * KERNEL_CLASSES)()
    _check(load().sph_profile_end(ctx, ms, cnt), "sph_profile_end")
    return {sph_kernel_class_name(k): (float(ms[k]), int(cnt[k])) for k in range(KERNEL_CLASSES)}


def sph_kernel_class_name(k: int) -> str:
    return load().sph_kernel_class_name(int(k)).decode()


def sph_set_density_rate(ctx, drho) -> None:
    """Dual-criteria integrator: the carried d rho/dt ([n], caller order)."""
    keep = []
    _check(load().sph_set_density_rate(ctx, _ptr(drho, keep, np.float64)), "sph_set_density_rate")


def sph_get_density_rate(ctx, out) -> None:
    keep = []
    _check(load().sph_get_density_rate(ctx, _ptr(out, keep, np.float64)), "sph_get_density_rate")


def sph_fma_peak(precision: int, blocks: int, iters: int, sink, stream=None) -> float:
    """Enqueue the FMA-throughput launch on ``stream`` (torch's current
    stream by default) into the device tensor ``sink`` (blocks * 256 float32
    or float64 elements) and return its floating-point operations; the
    caller times it with CUDA events on that stream."""
    import torch
    dtype = torch.float32 if precision == 32 else torch.float64
    if not (sink.is_cuda and sink.dtype == dtype and sink.numel() >= blocks * 256):
        raise ValueError("sink must be a CUDA %s tensor of at least blocks * 256 elements" % dtype)
    if stream is None:
        stream = torch.cuda.current_stream(sink.device)
    flops = ctypes.c_double(0.0)
    _check(load().sph_fma_peak(int(precision), int(blocks), int(iters), ctypes.c_void_p(sink.data_ptr()),
                               ctypes.c_void_p(stream.cuda_stream), ctypes.byref(flops)), "sph_fma_peak")
    return flops.value


NOALLOC_MAX_PARTICLES = 65536


def sph_density_noalloc(params: SphParams, n: int, x, h, m, kind, sigma0, rho, stream_ptr: int) -> None:
    """Density pass (FP64) into ``rho`` without any device allocation: for
    callers that cannot give the library a workspace (a host framework that
    owns all device memory, or a real-time loop where cudaMalloc could stall
    the device).  x, h, m, kind, sigma0 and rho are contiguous CUDA tensors
    (kind and sigma0 may be None); the library's fixed scratch limits n to
    NOALLOC_MAX_PARTICLES.  Calls that overlap on the GPU race on that scratch."""
    def dp(t):
        if t is None:
            return None
        assert t.is_cuda and t.is_contiguous()
        return _vp(t.data_ptr())
    _check(load().sph_density_noalloc(ctypes.byref(params), int(n), dp(x), dp(h), dp(m), dp(kind), dp(sigma0),
                                      dp(rho), _vp(stream_ptr)), "sph_density_noalloc")


def _p64(t, keep):
    """Pointer to a contiguous float64 array (numpy or torch, host or CUDA)."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        assert t.dtype.is_floating_point and t.element_size() == 8 and t.is_contiguous()
        return _vp(t.data_ptr())
    arr = np.ascontiguousarray(t, dtype=np.float64)
    keep.append(arr)
    return _vp(arr.ctypes.data)


def sph_step_adjoint(ctx, x0, v0, a0, dr0, nsteps: int, xbar, vbar, abar, drbar) -> float:
    """Reverse of ``nsteps`` steps from the checkpoint (x0, v0, a0, dr0).
    xbar, vbar, abar, drbar ([n][3] float64, numpy or torch, written in place)
    hold the cotangents of the state after the segment on entry and those of
    the checkpoint on return.  Returns d/d(eta) over the segment."""
    keep = []
    eta = ctypes.c_double(0.0)
    for t in (xbar, vbar, abar, drbar):
        if not hasattr(t, "data_ptr"):
            assert isinstance(t, np.ndarray) and t.flags["C_CONTIGUOUS"] and t.dtype == np.float64
    ptr = lambda t: _p64(t, keep) if hasattr(t, "data_ptr") else _vp(t.ctypes.data)
    _check(load().sph_step_adjoint(ctx, _p64(x0, keep), _p64(v0, keep), _p64(a0, keep), _p64(dr0, keep),
                                   int(nsteps), ptr(xbar), ptr(vbar), ptr(abar), ptr(drbar), ctypes.byref(eta)),
           "sph_step_adjoint")
    return eta.value


def sph_force_pass_adjoint(ctx, x, v, abar, drbar, xbar, vbar) -> float:
    """Reverse of the initial force pass on (x, v): ADD the cotangents of x
    and v to xbar, vbar (in place) given those of a and dr; returns
    d/d(eta)."""
    keep = []
    eta = ctypes.c_double(0.0)
    ptr = lambda t: _p64(t, keep) if hasattr(t, "data_ptr") else _vp(t.ctypes.data)
    _check(load().sph_force_pass_adjoint(ctx, _p64(x, keep), _p64(v, keep), _p64(abar, keep), _p64(drbar, keep),
                                         ptr(xbar), ptr(vbar), ctypes.byref(eta)), "sph_force_pass_adjoint")
    return eta.value


# ------------------------------------------------------------------ convenience

def params_from_case(case: dict, precision: int = 64, **kw) -> SphParams:
    """sph_params for a case dict from ``cases`` (paper constants by default)."""
    p = sph_default_params()
    p.dim = int(case["dim"])
    p.precision = int(precision)
    for d in range(3):
        p.periodic[d] = int(case["periodic"][d])
        p.lo[d] = float(case["lo"][d])
        p.L[d] = float(case["L"][d])
        p.g[d] = float(case.get("g", (0.0, 0.0, 0.0))[d])
    p.rho0, p.c0, p.eta = float(case["rho0"]), float(case["c"]), float(case["eta"])
    p.h_min, p.h_max, p.u_ref = float(case["h_min"]), float(case["h_max"]), float(case["u_ref"])
    for k, val in kw.items():
        if not hasattr(p, k):
            raise AttributeError("sph_params has no field %r" % k)
        setattr(p, k, val)
    return p


class Simulation:
    """One libsphtv context on the current CUDA device.

    torch provides the workspace (``sph_query_workspace`` bytes) and the
    stream (torch's current stream unless one is given)."""

    def __init__(self, case: dict, precision: int = 64, stream=None, **param_overrides):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libsphtv needs a CUDA device; none is available")
        load()
        self.case = case
        self.n = int(case["n"])
        self.params = params_from_case(case, precision, **param_overrides)
        self.nbytes = sph_query_workspace(self.params, self.n)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.ctx = sph_create(self.params, self.n, self.workspace.data_ptr(), self.nbytes, self.stream.cuda_stream)

    def set_state(self, x=None, v=None, a=None, dr=None, sigma0=None, drho=None):
        c = self.case
        sph_set_state(self.ctx, c["x"] if x is None else x, c["v"] if v is None else v, a, dr, c["h"], c["m"],
                      c.get("kind"), c.get("vw"), sigma0)
        if drho is not None:
            sph_set_density_rate(self.ctx, drho)

    def density_rate(self):
        out = np.zeros(self.n)
        sph_get_density_rate(self.ctx, out)
        return out

    def build_cells(self):
        sph_build_cells(self.ctx)

    def step(self, n: int = 1):
        sph_step(self.ctx, n)

    def set_dt(self, dt: float):
        sph_set_dt(self.ctx, dt)

    def get_state(self):
        n = self.n
        out = {k: np.zeros((n, 3)) for k in ("x", "v", "a", "dr")}
        out["rho"] = np.zeros(n)
        sph_get_state(self.ctx, out["x"], out["v"], out["a"], out["dr"], out["rho"])
        return out

    def diag(self) -> dict:
        return sph_get_diag(self.ctx).as_dict()

    def sync(self):
        sph_sync(self.ctx)

    def launches(self) -> int:
        return sph_launch_count(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            sph_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


class Rollout:
    """Differentiable rollout through libsphtv: (x0, v0, nu) -> (x_T, v_T).

    Forward: initial force pass on (x0, v0), then ``nsteps`` kick-drift-kick
    steps of the context's fixed dt, keeping the state every ``every`` steps
    (device FP64 tensors).  Backward: the library's hand-written adjoint,
    segment by segment from the last checkpoint (each segment is replayed
    from its checkpoint inside sph_step_adjoint), then the adjoint of the
    initial force pass; d/d(nu) = rho0 d/d(eta).  Neighbour sets and dt are
    frozen per step.  Use ``Rollout.apply(x0, v0, nu, sim, nsteps, every)``
    with a Simulation created with fixed_dt > 0 and adjoint_steps >= every.
    """

    @staticmethod
    def _function():
        import torch

        class _Rollout(torch.autograd.Function):
            @staticmethod
            def forward(fctx, x0, v0, nu, sim, nsteps, every):
                dev = sim.device
                x0d = x0.detach().to(device=dev, dtype=torch.float64).contiguous()
                v0d = v0.detach().to(device=dev, dtype=torch.float64).contiguous()
                sph_set_eta(sim.ctx, float(nu) * sim.params.rho0)
                c = sim.case
                sph_set_state(sim.ctx, x0d, v0d, None, None, c["h"], c["m"], c.get("kind"), c.get("vw"), None)
                sph_build_cells(sim.ctx)
                ckpts = []
                done = 0
                while done < nsteps:
                    seg = min(every, nsteps - done)
                    st = {k: torch.empty((sim.n, 3), dtype=torch.float64, device=dev) for k in ("x", "v", "a", "dr")}
                    sph_get_state(sim.ctx, st["x"], st["v"], st["a"], st["dr"], None)
                    ckpts.append((st, seg))
                    sph_step(sim.ctx, seg)
                    done += seg
                xT = torch.empty((sim.n, 3), dtype=torch.float64, device=dev)
                vT = torch.empty_like(xT)
                sph_get_state(sim.ctx, xT, vT, None, None, None)
                fctx.sim, fctx.ckpts, fctx.x0, fctx.v0 = sim, ckpts, x0d, v0d
                fctx.in_dev, fctx.in_dtype = x0.device, x0.dtype
                return xT, vT

            @staticmethod
            def backward(fctx, gx, gv):
                sim = fctx.sim
                dev = sim.device
                z = lambda g: (torch.zeros((sim.n, 3), dtype=torch.float64, device=dev) if g is None
                               else g.detach().to(device=dev, dtype=torch.float64).contiguous().clone())
                xb, vb = z(gx), z(gv)
                ab = torch.zeros_like(xb)
                drb = torch.zeros_like(xb)
                etab = 0.0
                for st, seg in reversed(fctx.ckpts):
                    etab += sph_step_adjoint(sim.ctx, st["x"], st["v"], st["a"], st["dr"], seg, xb, vb, ab, drb)
                etab += sph_force_pass_adjoint(sim.ctx, fctx.x0, fctx.v0, ab, drb, xb, vb)
                gnu = torch.tensor(etab * sim.params.rho0, dtype=torch.float64)
                return (xb.to(fctx.in_dev, fctx.in_dtype), vb.to(fctx.in_dev, fctx.in_dtype), gnu, None, None, None)

        return _Rollout

    _fn = None

    @classmethod
    def apply(cls, x0, v0, nu, sim, nsteps: int, every: int):
        if cls._fn is None:
            cls._fn = cls._function()
        return cls._fn.apply(x0, v0, nu, sim, nsteps, every)

