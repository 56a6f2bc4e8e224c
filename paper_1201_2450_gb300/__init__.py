"""GB300-native temporal non-local means (TNLM) 4D cone-beam CT.

Thin ctypes binding of ``libtnlm.so`` (see ``include/tnlm.h``): the functions
below carry the C-ABI names and only marshal arguments -- every arithmetic
step runs in the library's CUDA kernels.  PyTorch supplies device memory and
streams.  If the library has not been built, every call raises; there is no
CPU fallback.

    import paper_1201_2450_gb300 as tnlm
    tnlm.build()                                  # nvcc, sm_103a, in-tree
    geom = tnlm.tnlm_create_geometry(desc)        # desc: dict (see synth.make_geometry)
    proj = tnlm.tnlm_project(geom, vol)           # vol: cuda float32 [Np, nz, ny, nx]
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass

import numpy as np
import torch

from ._build import LIB as _LIB_PATH
from ._build import build

__all__ = [
    "build", "TnlmError", "Params", "Geometry", "tnlm_create_geometry", "tnlm_project", "tnlm_backproject",
    "tnlm_weights", "tnlm_gauss_jacobi", "tnlm_reconstruct", "tnlm_enhance", "tnlm_enhance_noalloc",
    "tnlm_operator_norm", "tnlm_cgls", "tnlm_fdk", "tnlm_gauss_jacobi_bf16", "tnlm_enhance_bf16",
    "tnlm_energy_grad", "tnlm_energy_grad_weights", "tnlm_energy_grad_bf16", "TNLMEnergy", "tnlm_reconstruct_batch", "BatchPlan", "tnlm_reconstruct_bf16",
    "tnlm_autotune", "tnlm_autotune_sweep", "tnlm_set_launch_shapes", "tnlm_get_launch_shapes", "tnlm_set_sweep_shape",
    "reconstruct_host", "library_path", "tnlm_peak_probe", "tnlm_gauss_jacobi_range", "tnlm_p1",
    "tnlm_reconstruct_fp16", "tnlm_enhance_fp16", "tnlm_gauss_jacobi_fp16", "tnlm_energy_grad_fp16",
    "tnlm_gauss_jacobi_pairs",
]

_lock = threading.Lock()
_lib = None


class TnlmError(RuntimeError):
    def __init__(self, status: int, func: str, detail: str):
        self.status = status
        super().__init__(f"{func} failed with status {status} ({_STATUS.get(status, '?')}): {detail}")


_STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "out of device memory", 4: "timeout",
           5: "not implemented"}


class _Desc(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
        ("cx", C.c_double), ("cy", C.c_double), ("cz", C.c_double),
        ("nu", C.c_int), ("nv", C.c_int),
        ("du", C.c_double), ("dv", C.c_double),
        ("u_off", C.c_double), ("v_off", C.c_double),
        ("sad", C.c_double), ("sdd", C.c_double),
        ("n_phases", C.c_int),
        ("n_views", C.POINTER(C.c_int)),
        ("angles_rad", C.POINTER(C.c_double)),
    ]


class _Params(C.Structure):
    _fields_ = [("d", C.c_int), ("M", C.c_int), ("h", C.c_float), ("mu", C.c_float), ("tau", C.c_float),
                ("n_outer", C.c_int), ("n_inner", C.c_int), ("clip_nonneg", C.c_int), ("gj_start", C.c_int),
                ("n_gj", C.c_int), ("p1_solver", C.c_int)]


@dataclass
class Params:
    """TNLM-R / TNLM-E parameters (mirror of ``tnlm_params``)."""
    d: int = 1
    M: int = 2
    h: float = 0.02
    mu: float = 1.0
    tau: float = 0.0
    n_outer: int = 1
    n_inner: int = 1
    clip_nonneg: int = 1
    gj_start: int = 0
    n_gj: int = 1
    p1_solver: int = 0

    def _c(self) -> _Params:
        return _Params(self.d, self.M, self.h, self.mu, self.tau, self.n_outer, self.n_inner, self.clip_nonneg,
                       self.gj_start, self.n_gj, self.p1_solver)


def library_path() -> str:
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"{_LIB_PATH} is missing: build it with paper_1201_2450_gb300.build() "
                               "(this package has no CPU fallback)")
        lib = C.CDLL(_LIB_PATH)
        vp, i, f, sz = C.c_void_p, C.c_int, C.c_float, C.c_size_t
        sig = {
            "tnlm_create_geometry": (i, [C.POINTER(_Desc), C.POINTER(vp)]),
            "tnlm_destroy_geometry": (None, [vp]),
            "tnlm_project": (i, [vp, vp, vp, vp]),
            "tnlm_backproject": (i, [vp, vp, vp, f, f, vp]),
            "tnlm_weights": (i, [i, i, i, i, vp, i, i, f, vp, sz, vp]),
            "tnlm_gauss_jacobi": (i, [i, i, i, i, vp, vp, vp, vp, i, i, f, f, i, vp]),
            "tnlm_gauss_jacobi_range": (i, [i, i, i, i, i, i, vp, vp, vp, vp, i, i, f, f, i, vp]),
            "tnlm_gauss_jacobi_pairs": (i, [i, i, i, i, vp, vp, vp, vp, i, i, f, f, i, vp]),
            "tnlm_set_batch_sweep_mode": (i, [i]),
            "tnlm_p1": (i, [vp, vp, vp, vp, C.POINTER(_Params), vp, vp]),
            "tnlm_reconstruct": (i, [vp, vp, vp, C.POINTER(_Params), vp, vp]),
            "tnlm_reconstruct_host": (i, [vp, vp, vp, vp, vp, C.POINTER(_Params), vp, vp]),
            "tnlm_enhance": (i, [i, i, i, i, vp, vp, C.POINTER(_Params), vp]),
            "tnlm_enhance_noalloc": (i, [i, i, i, i, vp, vp, C.POINTER(_Params), vp]),
            "tnlm_operator_norm": (i, [vp, vp, i, C.POINTER(C.c_double), vp]),
            "tnlm_cgls": (i, [vp, vp, vp, i, vp, vp]),
            "tnlm_fdk": (i, [vp, vp, vp, vp]),
            "tnlm_gauss_jacobi_bf16": (i, [i, i, i, i, vp, vp, vp, vp, i, i, f, f, i, vp]),
            "tnlm_energy_grad": (i, [vp, vp, vp, vp, C.POINTER(_Params), C.POINTER(C.c_double), vp, vp]),
            "tnlm_energy_grad_weights": (i, [i, i, i, i, vp, vp, i, i, f, vp, vp]),
            "tnlm_energy_grad_bf16": (i, [vp, vp, vp, vp, C.POINTER(_Params), C.POINTER(C.c_double), vp, vp]),
            "tnlm_reconstruct_batch": (i, [i, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(_Params), vp]),
            "tnlm_batch_plan_create": (i, [i, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(_Params),
                                           C.POINTER(vp)]),
            "tnlm_batch_plan_run": (i, [vp, i, vp]),
            "tnlm_batch_plan_create_bf16": (i, [i, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(_Params),
                                                C.POINTER(vp)]),
            "tnlm_reconstruct_bf16": (i, [vp, vp, vp, C.POINTER(_Params), vp, vp]),
            "tnlm_batch_plan_destroy": (None, [vp]),
            "tnlm_autotune": (i, [vp, C.POINTER(_Params), C.POINTER(C.c_int), vp]),
            "tnlm_autotune_sweep": (i, [i, i, i, i, i, i, f, i, C.POINTER(C.c_int), vp]),
            "tnlm_set_launch_shapes": (i, [vp, i, i, i]),
            "tnlm_get_launch_shapes": (i, [vp, C.POINTER(C.c_int)]),
            "tnlm_set_sweep_shape": (i, [i, i, i, i]),
            "tnlm_enhance_bf16": (i, [i, i, i, i, vp, vp, C.POINTER(_Params), vp]),
            "tnlm_enhance_fp16": (i, [i, i, i, i, vp, vp, C.POINTER(_Params), vp]),
            "tnlm_gauss_jacobi_fp16": (i, [i, i, i, i, vp, vp, vp, vp, i, i, f, f, i, vp]),
            "tnlm_energy_grad_fp16": (i, [vp, vp, vp, vp, C.POINTER(_Params), C.POINTER(C.c_double), vp, vp]),
            "tnlm_batch_plan_create_fp16": (i, [i, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(_Params),
                                                C.POINTER(vp)]),
            "tnlm_reconstruct_fp16": (i, [vp, vp, vp, C.POINTER(_Params), vp, vp]),
            "tnlm_set_stage_timing": (i, [vp, i]),
            "tnlm_peak_probe": (i, [i, i, i, vp, C.POINTER(C.c_double), vp]),
            "tnlm_test_fail_allocations": (i, [i]),
            "tnlm_get_stage_timing": (i, [vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
            "tnlm_status_string": (C.c_char_p, [i]),
            "tnlm_last_error": (C.c_char_p, []),
            "tnlm_version": (i, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(status: int, func: str):
    if status != 0:
        raise TnlmError(status, func, _load().tnlm_last_error().decode(errors="replace"))


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _dev(t: torch.Tensor, name: str, device: torch.device | None = None, shape=None,
         dtype=torch.float32) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, expected {device}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.data_ptr()


class Geometry:
    """Owns a ``tnlm_geometry`` handle created on the current CUDA device."""

    def __init__(self, desc: dict):
        lib = _load()
        self.desc = dict(desc)
        self._nviews = np.ascontiguousarray(np.asarray(desc["nviews"], dtype=np.int32))
        self._angles = np.ascontiguousarray(np.asarray(desc["angles"], dtype=np.float64))
        d = _Desc()
        for k in ("nx", "ny", "nz", "nu", "nv"):
            setattr(d, k, int(desc[k]))
        for k in ("dx", "dy", "dz", "cx", "cy", "cz", "du", "dv", "u_off", "v_off", "sad", "sdd"):
            setattr(d, k, float(desc.get(k, 0.0)))
        d.n_phases = int(self._nviews.size)
        d.n_views = self._nviews.ctypes.data_as(C.POINTER(C.c_int))
        d.angles_rad = self._angles.ctypes.data_as(C.POINTER(C.c_double))
        if self._angles.size != int(self._nviews.sum()):
            raise ValueError("angles must hold sum(nviews) entries")
        h = C.c_void_p()
        self._h = None
        _check(lib.tnlm_create_geometry(C.byref(d), C.byref(h)), "tnlm_create_geometry")
        self._h = h
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.np = d.n_phases
        self.vol_shape = (d.n_phases, d.nz, d.ny, d.nx)
        self.proj_shape = (int(self._nviews.sum()), d.nv, d.nu)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _load().tnlm_destroy_geometry(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stage_timing(self, enable: bool):
        _check(_load().tnlm_set_stage_timing(self._h, int(enable)), "tnlm_set_stage_timing")

    def stage_timing(self):
        ms = (C.c_double * 3)()
        n = (C.c_longlong * 3)()
        _check(_load().tnlm_get_stage_timing(self._h, ms, n), "tnlm_get_stage_timing")
        return list(ms), list(n)


def tnlm_create_geometry(desc: dict) -> Geometry:
    return Geometry(desc)


def tnlm_project(geom: Geometry, vol: torch.Tensor, proj: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """proj = P vol (exact radiological path, all phases)."""
    if proj is None:
        proj = torch.empty(geom.proj_shape, dtype=torch.float32, device=geom.device)
    _check(_load().tnlm_project(geom.handle, _dev(vol, "vol", geom.device, geom.vol_shape),
                                _dev(proj, "proj", geom.device, geom.proj_shape), _stream(stream)), "tnlm_project")
    return proj


def tnlm_backproject(geom: Geometry, proj: torch.Tensor, vol: torch.Tensor | None = None, alpha: float = 1.0,
                     beta: float = 0.0, stream=None) -> torch.Tensor:
    """vol = beta vol + alpha P^T proj."""
    if vol is None:
        vol = torch.empty(geom.vol_shape, dtype=torch.float32, device=geom.device)
        beta = 0.0
    _check(_load().tnlm_backproject(geom.handle, _dev(proj, "proj", geom.device, geom.proj_shape),
                                    _dev(vol, "vol", geom.device, geom.vol_shape), alpha, beta, _stream(stream)),
           "tnlm_backproject")
    return vol


def tnlm_weights(wsrc: torch.Tensor, d: int, M: int, h: float, out: torch.Tensor | None = None,
                 stream=None) -> torch.Tensor:
    """Normalised Eq. 9 weights, [Np][2][nz][ny][nx][(2M+1)^3]."""
    np_, nz, ny, nx = wsrc.shape
    W = (2 * M + 1) ** 3
    if out is None:
        out = torch.empty((np_, 2, nz, ny, nx, W), dtype=torch.float32, device=wsrc.device)
    _check(_load().tnlm_weights(nx, ny, nz, np_, _dev(wsrc, "wsrc"), d, M, h, _dev(out, "w_out", wsrc.device),
                                out.numel(), _stream(stream)), "tnlm_weights")
    return out


def tnlm_gauss_jacobi(wsrc: torch.Tensor, vals: torch.Tensor, g: torch.Tensor, d: int, M: int, h: float, mu: float,
                      clip: int = 0, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """One Eq. 8 sweep with weights (Eq. 9) from wsrc."""
    np_, nz, ny, nx = wsrc.shape
    if out is None:
        out = torch.empty_like(wsrc)
    dev = wsrc.device
    _check(_load().tnlm_gauss_jacobi(nx, ny, nz, np_, _dev(wsrc, "wsrc"), _dev(vals, "vals", dev, wsrc.shape),
                                     _dev(g, "g", dev, wsrc.shape), _dev(out, "f_out", dev, wsrc.shape), d, M, h,
                                     mu, int(clip), _stream(stream)), "tnlm_gauss_jacobi")
    return out


def tnlm_gauss_jacobi_pairs(wsrc: torch.Tensor, vals: torch.Tensor, g: torch.Tensor, d: int, M: int, h: float,
                            mu: float, clip: int = 0, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """One Eq. 8 sweep with each phase pair's patch distances computed once
    (Sec. 2.4); the same result as tnlm_gauss_jacobi to rounding."""
    np_, nz, ny, nx = wsrc.shape
    if out is None:
        out = torch.empty_like(wsrc)
    dev = wsrc.device
    _check(_load().tnlm_gauss_jacobi_pairs(nx, ny, nz, np_, _dev(wsrc, "wsrc"), _dev(vals, "vals", dev, wsrc.shape),
                                           _dev(g, "g", dev, wsrc.shape), _dev(out, "f_out", dev, wsrc.shape), d, M,
                                           h, mu, int(clip), _stream(stream)), "tnlm_gauss_jacobi_pairs")
    return out


def tnlm_gauss_jacobi_range(wsrc: torch.Tensor, vals: torch.Tensor, g: torch.Tensor, out: torch.Tensor, p0: int,
                            n_out: int, d: int, M: int, h: float, mu: float, clip: int = 0, stream=None):
    """One Eq. 8 sweep of the output phases p0 .. p0 + n_out - 1 of arrays of
    wsrc.shape[0] phases (ring neighbours (i +- 1) mod that count) into out."""
    np_, nz, ny, nx = wsrc.shape
    dev = wsrc.device
    _check(_load().tnlm_gauss_jacobi_range(nx, ny, nz, np_, int(p0), int(n_out), _dev(wsrc, "wsrc"),
                                           _dev(vals, "vals", dev, wsrc.shape), _dev(g, "g", dev, wsrc.shape),
                                           _dev(out, "f_out", dev, wsrc.shape), d, M, h, mu, int(clip),
                                           _stream(stream)), "tnlm_gauss_jacobi_range")
    return out


def tnlm_p1(geom: Geometry, y: torch.Tensor, f: torch.Tensor, g: torch.Tensor, params: Params, report: bool = False,
            stream=None):
    """(P1) of one FBS iteration from f into g (params.n_inner gradient steps or
    CGLS iterations); returns the residual norms before each step, or None."""
    rep = np.zeros(params.n_inner, np.float64) if report else None
    p = params._c()
    _check(_load().tnlm_p1(geom.handle, _dev(y, "y", geom.device, geom.proj_shape),
                           _dev(f, "f", geom.device, geom.vol_shape), _dev(g, "g", geom.device, geom.vol_shape),
                           C.byref(p), rep.ctypes.data if rep is not None else None, _stream(stream)), "tnlm_p1")
    return rep


def tnlm_reconstruct(geom: Geometry, y: torch.Tensor, f: torch.Tensor, params: Params, report: bool = False,
                     stream=None):
    """TNLM-R in place on f; returns (f, report or None)."""
    rep = np.zeros((params.n_outer, params.n_inner), np.float64) if report else None
    p = params._c()
    _check(_load().tnlm_reconstruct(geom.handle, _dev(y, "y", geom.device, geom.proj_shape),
                                    _dev(f, "f", geom.device, geom.vol_shape), C.byref(p),
                                    rep.ctypes.data if rep is not None else None, _stream(stream)),
           "tnlm_reconstruct")
    return f, rep


def _batch_args(geoms, ys, fs, params, dtype=torch.float32):
    n = len(geoms)
    if not (len(ys) == len(fs) == len(params) == n):
        raise ValueError("geoms, ys, fs and params must have the same length")
    G = (C.c_void_p * n)(*[g.handle.value for g in geoms])
    Y = (C.c_void_p * n)(*[_dev(y, "y", g.device, g.proj_shape, dtype) for g, y in zip(geoms, ys)])
    F = (C.c_void_p * n)(*[_dev(f, "f", g.device, g.vol_shape, dtype) for g, f in zip(geoms, fs)])
    P = (_Params * n)(*[p._c() for p in params])
    return n, G, Y, F, P


def tnlm_reconstruct_batch(geoms, ys, fs, params, stream=None):
    """TNLM-R on independent problems in one graph replayed n_outer times;
    every f is updated in place."""
    n, G, Y, F, P = _batch_args(geoms, ys, fs, params)
    _check(_load().tnlm_reconstruct_batch(n, G, Y, F, P, _stream(stream)), "tnlm_reconstruct_batch")
    return fs


def _reconstruct16(name, dtype, geom, y, f, params, report, stream):
    rep = np.zeros((params.n_outer, params.n_inner), np.float64) if report else None
    p = params._c()
    _check(getattr(_load(), name)(geom.handle, _dev(y, "y", geom.device, geom.proj_shape, dtype),
                                  _dev(f, "f", geom.device, geom.vol_shape, dtype), C.byref(p),
                                  rep.ctypes.data if rep is not None else None, _stream(stream)), name)
    return f, rep


def tnlm_reconstruct_bf16(geom: Geometry, y: torch.Tensor, f: torch.Tensor, params: Params, report: bool = False,
                          stream=None):
    """TNLM-R in place on bfloat16 f from bfloat16 y, FP32 arithmetic;
    returns (f, report or None)."""
    return _reconstruct16("tnlm_reconstruct_bf16", torch.bfloat16, geom, y, f, params, report, stream)


def tnlm_reconstruct_fp16(geom: Geometry, y: torch.Tensor, f: torch.Tensor, params: Params, report: bool = False,
                          stream=None):
    """TNLM-R in place on float16 f from float16 y, FP32 arithmetic;
    returns (f, report or None)."""
    return _reconstruct16("tnlm_reconstruct_fp16", torch.float16, geom, y, f, params, report, stream)


def tnlm_autotune(geom: Geometry, params: Params, stream=None) -> dict:
    """Time the compiled launch shapes on this problem and keep the fastest
    (projector and transpose shapes in the handle, the FP32 sweep shape for
    (d, M) process-wide).  Results do not depend on the choice."""
    out = (C.c_int * 4)()
    p = params._c()
    _check(_load().tnlm_autotune(geom.handle, C.byref(p), out, _stream(stream)), "tnlm_autotune")
    return {"projector_rows": out[0], "transpose_cells": out[1], "transpose_rows": out[2], "sweep_shape": out[3]}


def _storage(bf16, fp16) -> int:
    return 2 if fp16 else (1 if bf16 else 0)


def tnlm_autotune_sweep(shape, d: int, M: int, h: float, bf16: bool = False, stream=None, fp16: bool = False) -> int:
    """Tune the box-sum sweep for a [N_p, nz, ny, nx] problem (FP32, BF16 or
    FP16 storage); returns the shape index."""
    np_, nz, ny, nx = shape
    out = C.c_int()
    _check(_load().tnlm_autotune_sweep(nx, ny, nz, np_, d, M, h, _storage(bf16, fp16), C.byref(out), _stream(stream)),
           "tnlm_autotune_sweep")
    return out.value


def tnlm_set_launch_shapes(geom: Geometry, projector_rows: int, transpose_cells: int, transpose_rows: int):
    _check(_load().tnlm_set_launch_shapes(geom.handle, projector_rows, transpose_cells, transpose_rows),
           "tnlm_set_launch_shapes")


def tnlm_get_launch_shapes(geom: Geometry) -> dict:
    """The handle's launch shapes as they run now (projector code 4 while a
    table shape has no tables)."""
    out = (C.c_int * 3)()
    _check(_load().tnlm_get_launch_shapes(geom.handle, out), "tnlm_get_launch_shapes")
    return {"projector_rows": out[0], "transpose_cells": out[1], "transpose_rows": out[2]}


def tnlm_set_sweep_shape(d: int, M: int, bf16: bool, shape: int, fp16: bool = False):
    _check(_load().tnlm_set_sweep_shape(d, M, _storage(bf16, fp16), shape), "tnlm_set_sweep_shape")


class BatchPlan:
    """One FBS iteration of every problem captured once (tnlm_batch_plan_*);
    run(k) replays it k times, updating every f in place.  The plan keeps
    references to the geometries and tensors it was built on."""

    def __init__(self, geoms, ys, fs, params, grouped: bool = False):
        """grouped: the sweeps of all problems in one persistent launch
        (tnlm_set_batch_sweep_mode(1) while the plan is made)."""
        dtype = fs[0].dtype if len(fs) > 0 else torch.float32
        n, G, Y, F, P = _batch_args(geoms, ys, fs, params, dtype)
        self._keep = (list(geoms), list(ys), list(fs))
        self.handle = C.c_void_p()
        create = {torch.bfloat16: _load().tnlm_batch_plan_create_bf16,
                  torch.float16: _load().tnlm_batch_plan_create_fp16}.get(dtype, _load().tnlm_batch_plan_create)
        _check(_load().tnlm_set_batch_sweep_mode(1 if grouped else 0), "tnlm_set_batch_sweep_mode")
        try:
            _check(create(n, G, Y, F, P, C.byref(self.handle)), "tnlm_batch_plan_create")
        finally:
            _load().tnlm_set_batch_sweep_mode(0)

    def run(self, n_iterations: int, stream=None):
        _check(_load().tnlm_batch_plan_run(self.handle, int(n_iterations), _stream(stream)), "tnlm_batch_plan_run")

    def close(self):
        if self.handle:
            _load().tnlm_batch_plan_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tnlm_enhance(g: torch.Tensor, params: Params, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """TNLM-E: f^(0) = g, params.n_outer sweeps."""
    np_, nz, ny, nx = g.shape
    if out is None:
        out = torch.empty_like(g)
    p = params._c()
    _check(_load().tnlm_enhance(nx, ny, nz, np_, _dev(g, "g"), _dev(out, "f", g.device, g.shape), C.byref(p),
                                _stream(stream)), "tnlm_enhance")
    return out


def tnlm_enhance_noalloc(g: torch.Tensor, params: Params, out: torch.Tensor, stream=None) -> torch.Tensor:
    """TNLM-E that allocates nothing on the device: the caller provides the
    output and the library's fixed 16 MiB scratch array holds the ping-pong
    image (at most 4 Mi voxels over all phases)."""
    np_, nz, ny, nx = g.shape
    p = params._c()
    _check(_load().tnlm_enhance_noalloc(nx, ny, nz, np_, _dev(g, "g"), _dev(out, "f", g.device, g.shape),
                                        C.byref(p), _stream(stream)), "tnlm_enhance_noalloc")
    return out


def tnlm_peak_probe(kind: int, blocks: int, iters: int, sink: torch.Tensor, stream=None) -> float:
    """Launch one throughput probe (0: FP32 FMA, 1: packed FP32x2 FMA, 2: ex2)
    on `stream`; returns the operations of the launch (FLOP for the FMA
    kinds, evaluations for ex2).  The caller times it with CUDA events."""
    ops = C.c_double(0.0)
    _check(_load().tnlm_peak_probe(int(kind), int(blocks), int(iters), _dev(sink, "sink"), C.byref(ops),
                                   _stream(stream)), "tnlm_peak_probe")
    return float(ops.value)


def tnlm_cgls(geom: Geometry, y: torch.Tensor, x: torch.Tensor, n_iter: int, report: bool = False, stream=None):
    """(P1) by CGLS, phase by phase, in place on x; returns (x, residual norms or None)."""
    rep = np.zeros(n_iter + 1, np.float64) if report else None
    _check(_load().tnlm_cgls(geom.handle, _dev(y, "y", geom.device, geom.proj_shape),
                             _dev(x, "x", geom.device, geom.vol_shape), n_iter,
                             rep.ctypes.data if rep is not None else None, _stream(stream)), "tnlm_cgls")
    return x, rep


def tnlm_fdk(geom: Geometry, proj: torch.Tensor, vol: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """FDK of every phase from its own views (full rotation, ref. 16)."""
    if vol is None:
        vol = torch.empty(geom.vol_shape, dtype=torch.float32, device=geom.device)
    _check(_load().tnlm_fdk(geom.handle, _dev(proj, "proj", geom.device, geom.proj_shape),
                            _dev(vol, "vol", geom.device, geom.vol_shape), _stream(stream)), "tnlm_fdk")
    return vol


def tnlm_gauss_jacobi_bf16(wsrc: torch.Tensor, vals: torch.Tensor, g: torch.Tensor, d: int, M: int, h: float,
                           mu: float, clip: int = 0, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """One Eq. 8 sweep on bfloat16 images with FP32 arithmetic."""
    np_, nz, ny, nx = wsrc.shape
    if out is None:
        out = torch.empty_like(wsrc)
    bf, dev = torch.bfloat16, wsrc.device
    _check(_load().tnlm_gauss_jacobi_bf16(nx, ny, nz, np_, _dev(wsrc, "wsrc", dtype=bf),
                                          _dev(vals, "vals", dev, wsrc.shape, bf), _dev(g, "g", dev, wsrc.shape, bf),
                                          _dev(out, "f_out", dev, wsrc.shape, bf), d, M, h, mu, int(clip),
                                          _stream(stream)), "tnlm_gauss_jacobi_bf16")
    return out


def tnlm_gauss_jacobi_fp16(wsrc: torch.Tensor, vals: torch.Tensor, g: torch.Tensor, d: int, M: int, h: float,
                           mu: float, clip: int = 0, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """One Eq. 8 sweep on float16 images with FP32 arithmetic."""
    np_, nz, ny, nx = wsrc.shape
    if out is None:
        out = torch.empty_like(wsrc)
    hf, dev = torch.float16, wsrc.device
    _check(_load().tnlm_gauss_jacobi_fp16(nx, ny, nz, np_, _dev(wsrc, "wsrc", dtype=hf),
                                          _dev(vals, "vals", dev, wsrc.shape, hf), _dev(g, "g", dev, wsrc.shape, hf),
                                          _dev(out, "f_out", dev, wsrc.shape, hf), d, M, h, mu, int(clip),
                                          _stream(stream)), "tnlm_gauss_jacobi_fp16")
    return out


def tnlm_enhance_fp16(g: torch.Tensor, params: Params, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """TNLM-E on float16 images with FP32 arithmetic."""
    np_, nz, ny, nx = g.shape
    if out is None:
        out = torch.empty_like(g)
    p = params._c()
    hf = torch.float16
    _check(_load().tnlm_enhance_fp16(nx, ny, nz, np_, _dev(g, "g", dtype=hf), _dev(out, "f", g.device, g.shape, hf),
                                     C.byref(p), _stream(stream)), "tnlm_enhance_fp16")
    return out


def tnlm_enhance_bf16(g: torch.Tensor, params: Params, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """TNLM-E on bfloat16 images with FP32 arithmetic."""
    np_, nz, ny, nx = g.shape
    if out is None:
        out = torch.empty_like(g)
    p = params._c()
    bf = torch.bfloat16
    _check(_load().tnlm_enhance_bf16(nx, ny, nz, np_, _dev(g, "g", dtype=bf), _dev(out, "f", g.device, g.shape, bf),
                                     C.byref(p), _stream(stream)), "tnlm_enhance_bf16")
    return out


def tnlm_energy_grad(geom: Geometry, y: torch.Tensor, f: torch.Tensor, a: torch.Tensor, params: Params,
                     grad: torch.Tensor | None = None, stream=None):
    """(E, grad E) of Eq. 1 with J of Eq. 2 and frozen Eq. 9 weights from a."""
    if grad is None:
        grad = torch.empty(geom.vol_shape, dtype=torch.float32, device=geom.device)
    E = C.c_double()
    p = params._c()
    _check(_load().tnlm_energy_grad(geom.handle, _dev(y, "y", geom.device, geom.proj_shape),
                                    _dev(f, "f", geom.device, geom.vol_shape), _dev(a, "a", geom.device, geom.vol_shape),
                                    C.byref(p), C.byref(E), _dev(grad, "grad", geom.device, geom.vol_shape),
                                    _stream(stream)), "tnlm_energy_grad")
    return E.value, grad


def tnlm_energy_grad_bf16(geom: Geometry, y: torch.Tensor, f: torch.Tensor, a: torch.Tensor, params: Params,
                          grad: torch.Tensor | None = None, stream=None):
    """tnlm_energy_grad on bfloat16 y, f and a; the gradient is FP32."""
    if grad is None:
        grad = torch.empty(geom.vol_shape, dtype=torch.float32, device=geom.device)
    E = C.c_double()
    p = params._c()
    b = torch.bfloat16
    _check(_load().tnlm_energy_grad_bf16(geom.handle, _dev(y, "y", geom.device, geom.proj_shape, b),
                                         _dev(f, "f", geom.device, geom.vol_shape, b),
                                         _dev(a, "a", geom.device, geom.vol_shape, b), C.byref(p), C.byref(E),
                                         _dev(grad, "grad", geom.device, geom.vol_shape), _stream(stream)),
           "tnlm_energy_grad_bf16")
    return E.value, grad


def tnlm_energy_grad_fp16(geom: Geometry, y: torch.Tensor, f: torch.Tensor, a: torch.Tensor, params: Params,
                          grad: torch.Tensor | None = None, stream=None):
    """tnlm_energy_grad on float16 y, f and a; the gradient is FP32."""
    if grad is None:
        grad = torch.empty(geom.vol_shape, dtype=torch.float32, device=geom.device)
    E = C.c_double()
    p = params._c()
    hf = torch.float16
    _check(_load().tnlm_energy_grad_fp16(geom.handle, _dev(y, "y", geom.device, geom.proj_shape, hf),
                                         _dev(f, "f", geom.device, geom.vol_shape, hf),
                                         _dev(a, "a", geom.device, geom.vol_shape, hf), C.byref(p), C.byref(E),
                                         _dev(grad, "grad", geom.device, geom.vol_shape), _stream(stream)),
           "tnlm_energy_grad_fp16")
    return E.value, grad


def tnlm_energy_grad_weights(f: torch.Tensor, a: torch.Tensor, d: int, M: int, h: float,
                             grad_a: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Gradient of 1/2 sum J (weights of Eq. 9 from a) with respect to a, f
    fixed: the weights differentiated."""
    np_, nz, ny, nx = f.shape
    if grad_a is None:
        grad_a = torch.empty_like(f)
    _check(_load().tnlm_energy_grad_weights(nx, ny, nz, np_, _dev(f, "f"), _dev(a, "a", f.device, f.shape), d, M, h,
                                            _dev(grad_a, "grad_a", f.device, f.shape), _stream(stream)),
           "tnlm_energy_grad_weights")
    return grad_a


class TNLMEnergy(torch.autograd.Function):
    """E(f, a) of Eq. 1 (J of Eq. 2 with the Eq. 9 weights computed from a)
    as an autograd function.  The forward pass computes the energy and its
    gradient in f with the library's kernels (projector, transpose, TNLM
    adjoint); the backward pass scales it, and when a requires a gradient it
    adds the gradient through the weights (tnlm_energy_grad_weights).
    Weights frozen: E = TNLMEnergy.apply(f, geom, y, a.detach(), params);
    weights differentiated (computed from f itself):
    E = TNLMEnergy.apply(f, geom, y, f, params)."""

    @staticmethod
    def forward(ctx, f, geom, y, a, params):
        fd, ad = f.detach().contiguous(), a.detach().contiguous()
        E, grad = tnlm_energy_grad(geom, y, fd, ad, params)
        ctx.save_for_backward(grad, fd, ad)
        ctx.params = params
        return torch.tensor(E, dtype=torch.float64, device=f.device)

    @staticmethod
    def backward(ctx, gE):
        grad, fd, ad = ctx.saved_tensors
        g = gE.to(grad.dtype)
        ga = None
        if ctx.needs_input_grad[3]:
            p = ctx.params
            ga = g * tnlm_energy_grad_weights(fd, ad, p.d, p.M, p.h)
        return (g * grad if ctx.needs_input_grad[0] else None, None, None, ga, None)


def tnlm_operator_norm(geom: Geometry, x: torch.Tensor, n_iter: int = 30, stream=None) -> float:
    """||P||^2 estimate (power iteration); x is overwritten."""
    L = C.c_double()
    _check(_load().tnlm_operator_norm(geom.handle, _dev(x, "x", geom.device, geom.vol_shape), n_iter, C.byref(L),
                                      _stream(stream)), "tnlm_operator_norm")
    return L.value


def _host(t: torch.Tensor, name: str, shape) -> int:
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise ValueError(f"{name} must be a host tensor")
    if t.dtype != torch.float32:
        raise ValueError(f"{name} must be torch.float32")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.data_ptr()


def reconstruct_host(geom: Geometry, y_host: torch.Tensor, f_host: torch.Tensor, params: Params,
                     y_dev: torch.Tensor | None = None, f_dev: torch.Tensor | None = None, stream=None,
                     report: bool = False):
    """TNLM-R on host buffers through tnlm_reconstruct_host: the copies to
    y_dev / f_dev, the run and the copy of f back into f_host, enqueued on the
    stream (pinned host memory lets the copies overlap the first projection).
    f_host holds the result once the stream has completed.  Returns the H2D
    and D2H byte counts (and the report when asked)."""
    if y_dev is None:
        y_dev = torch.empty(geom.proj_shape, dtype=torch.float32, device=geom.device)
    if f_dev is None:
        f_dev = torch.empty(geom.vol_shape, dtype=torch.float32, device=geom.device)
    rep = np.zeros((params.n_outer, params.n_inner), np.float64) if report else None
    p = params._c()
    _check(_load().tnlm_reconstruct_host(geom.handle, _host(y_host, "y_host", geom.proj_shape),
                                         _host(f_host, "f_host", geom.vol_shape),
                                         _dev(y_dev, "y_dev", geom.device, geom.proj_shape),
                                         _dev(f_dev, "f_dev", geom.device, geom.vol_shape), C.byref(p),
                                         rep.ctypes.data if rep is not None else None, _stream(stream)),
           "tnlm_reconstruct_host")
    counts = (y_host.numel() * 4 + f_host.numel() * 4, f_host.numel() * 4)
    return counts + (rep,) if report else counts
