"""FP64 CPU oracle of the TNLM 4D-CBCT method -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and
shares no code with it.

The C source (``tnlm_oracle.c``) restates the paper's definitions in double
precision; this module compiles it with gcc (``build()``) and wraps every
entry point with numpy arrays.  Geometry is passed as a plain dict with the
keys produced by ``paper_1201_2450_gb300.synth`` (nx, ny, nz, dx, dy, dz, cx,
cy, cz, nu, nv, du, dv, u_off, v_off, sad, sdd, nviews, angles).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tnlm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libtnlm_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libtnlm_oracle.so`` (gcc, OpenMP).

    ``-ffp-contract=off`` keeps the arithmetic identical on x86 and Arm (no
    fused multiply-add contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Geom(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
        ("cx", C.c_double), ("cy", C.c_double), ("cz", C.c_double),
        ("nu", C.c_int), ("nv", C.c_int),
        ("du", C.c_double), ("dv", C.c_double),
        ("u_off", C.c_double), ("v_off", C.c_double),
        ("sad", C.c_double), ("sdd", C.c_double),
        ("np", C.c_int),
        ("nviews", C.POINTER(C.c_int)),
        ("angles", C.POINTER(C.c_double)),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        G = C.POINTER(_Geom)
        i, d = C.c_int, C.c_double
        sig = {
            "ora_project": (None, [G, _dp, _dp]),
            "ora_backproject": (None, [G, _dp, _dp]),
            "ora_project_ray": (d, [G, _dp, i, i, i]),
            "ora_backproject_voxel": (d, [G, _dp, i, i, i, i]),
            "ora_power_norm": (d, [G, _dp, i]),
            "ora_chord": (d, [_dp, _dp, _dp, _dp]),
            "ora_ray": (None, [G, d, i, i, _dp, _dp]),
            "ora_weights": (None, [i, i, i, i, _dp, i, i, d, _dp]),
            "ora_gj_apply": (None, [i, i, i, i, _dp, i, _dp, _dp, d, i, _dp]),
            "ora_gj_voxel": (d, [i, i, i, i, _dp, _dp, _dp, i, i, i, i, i, i, d, d, i]),
            "ora_gj_sweep": (None, [i, i, i, i, _dp, _dp, _dp, i, i, d, d, i, _dp]),
            "ora_tnlm_energy": (d, [i, i, i, i, _dp, i, _dp]),
            "ora_fidelity": (d, [G, _dp, _dp]),
            "ora_reconstruct": (None, [G, _dp, _dp, d, i, i, d, d, i, i, i, i, i, i, C.c_void_p]),
            "ora_cgls": (None, [G, _dp, _dp, i, C.c_void_p]),
            "ora_fdk": (None, [G, _dp, _dp, C.c_void_p]),
            "ora_energy_grad": (d, [G, _dp, _dp, _dp, i, i, d, d, _dp]),
            "ora_energy_grad_a": (None, [i, i, i, i, _dp, _dp, i, i, d, _dp]),
            "ora_enhance": (None, [i, i, i, i, _dp, _dp, i, i, d, d, i, i]),
            "ora_num_threads": (i, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Geometry:
    """Owns the ctypes struct and the arrays it points into."""

    def __init__(self, desc: dict):
        self.desc = dict(desc)
        self._nviews = np.ascontiguousarray(np.asarray(desc["nviews"], dtype=np.int32))
        self._angles = _f64(desc["angles"])
        if self._angles.size != int(self._nviews.sum()):
            raise ValueError("angles must hold sum(nviews) entries")
        s = _Geom()
        for k in ("nx", "ny", "nz", "nu", "nv"):
            setattr(s, k, int(desc[k]))
        for k in ("dx", "dy", "dz", "cx", "cy", "cz", "du", "dv", "u_off", "v_off", "sad", "sdd"):
            setattr(s, k, float(desc.get(k, 0.0)))
        s.np = int(self._nviews.size)
        s.nviews = self._nviews.ctypes.data_as(C.POINTER(C.c_int))
        s.angles = self._angles.ctypes.data_as(C.POINTER(C.c_double))
        self.s = s
        self.np = s.np
        self.vol_shape = (s.np, s.nz, s.ny, s.nx)
        self.proj_shape = (int(self._nviews.sum()), s.nv, s.nu)

    @property
    def ref(self):
        return C.byref(self.s)


def project(geom: Geometry, f) -> np.ndarray:
    """P f for all phases (Eq. 1 data term), FP64."""
    lib = _load()
    f = _f64(f).reshape(geom.vol_shape)
    out = np.empty(geom.proj_shape, np.float64)
    lib.ora_project(geom.ref, f, out)
    return out


def backproject(geom: Geometry, proj) -> np.ndarray:
    """P^T proj (scatter of the Siddon segment lists), FP64."""
    lib = _load()
    proj = _f64(proj).reshape(geom.proj_shape)
    out = np.empty(geom.vol_shape, np.float64)
    lib.ora_backproject(geom.ref, proj, out)
    return out


def project_ray(geom: Geometry, f, view: int, iu: int, iv: int) -> float:
    return _load().ora_project_ray(geom.ref, _f64(f).reshape(geom.vol_shape), view, iu, iv)


def backproject_voxel(geom: Geometry, proj, phase: int, ix: int, iy: int, iz: int) -> float:
    """(P^T proj) at one voxel by the plain definition over every ray."""
    return _load().ora_backproject_voxel(geom.ref, _f64(proj).reshape(geom.proj_shape), phase, ix, iy, iz)


def power_norm(geom: Geometry, x0, n_iter: int = 50) -> float:
    """||P||_2^2 estimate by power iteration on P^T P started at x0."""
    x = _f64(x0).reshape(geom.vol_shape).copy()
    return _load().ora_power_norm(geom.ref, x, n_iter)


def chord(lo, hi, s, p) -> float:
    return _load().ora_chord(_f64(lo), _f64(hi), _f64(s), _f64(p))


def ray(geom: Geometry, theta: float, iu: int, iv: int):
    s = np.zeros(3)
    p = np.zeros(3)
    _load().ora_ray(geom.ref, theta, iu, iv, s, p)
    return s, p


def weights(a, d: int, M: int, h: float) -> np.ndarray:
    """Normalised Eq. 9 weights, shape [np][2][nz][ny][nx][(2M+1)^3]."""
    a = _f64(a)
    np_, nz, ny, nx = a.shape
    W = (2 * M + 1) ** 3
    out = np.empty((np_, 2, nz, ny, nx, W), np.float64)
    _load().ora_weights(nx, ny, nz, np_, a, d, M, h, out)
    return out


def gj_apply(w, M: int, vals, g, mu: float, clip: int = 0) -> np.ndarray:
    """Eq. 8 with the given weights (layout of ``weights``)."""
    vals = _f64(vals)
    np_, nz, ny, nx = vals.shape
    out = np.empty_like(vals)
    _load().ora_gj_apply(nx, ny, nz, np_, _f64(w), M, vals, _f64(g), mu, clip, out)
    return out


def gj_sweep(a, vals, g, d: int, M: int, h: float, mu: float, clip: int = 0) -> np.ndarray:
    """One sweep: weights from a (Eq. 9), update Eq. 8 from vals and g."""
    a = _f64(a)
    np_, nz, ny, nx = a.shape
    out = np.empty_like(a)
    _load().ora_gj_sweep(nx, ny, nz, np_, a, _f64(vals), _f64(g), d, M, h, mu, clip, out)
    return out


def gj_voxel(a, vals, g, phase: int, ix: int, iy: int, iz: int, d: int, M: int, h: float, mu: float,
             clip: int = 0) -> float:
    a = _f64(a)
    np_, nz, ny, nx = a.shape
    return _load().ora_gj_voxel(nx, ny, nz, np_, a, _f64(vals), _f64(g), phase, ix, iy, iz, d, M, h, mu, clip)


def tnlm_energy(w, M: int, f) -> float:
    """sum_i J[f_i, f_{i+1}] (Eq. 2 over the window) with frozen weights."""
    f = _f64(f)
    np_, nz, ny, nx = f.shape
    return _load().ora_tnlm_energy(nx, ny, nz, np_, _f64(w), M, f)


def energy_grad(geom: Geometry, y, f, a, d: int, M: int, h: float, mu: float):
    """(E, grad E) of Eq. 1 with J of Eq. 2 and frozen weights from a."""
    grad = np.empty(geom.vol_shape, np.float64)
    E = _load().ora_energy_grad(geom.ref, _f64(y).reshape(geom.proj_shape), _f64(f).reshape(geom.vol_shape),
                                _f64(a).reshape(geom.vol_shape), d, M, h, mu, grad)
    return E, grad


def energy_grad_a(f, a, d: int, M: int, h: float):
    """Gradient of 1/2 sum_i J[f_i, f_{i+1}] (weights of Eq. 9 from a) with
    respect to a, f held fixed: the weights differentiated."""
    np_, nz, ny, nx = np.shape(f)
    g = np.empty((np_, nz, ny, nx), np.float64)
    _load().ora_energy_grad_a(nx, ny, nz, np_, _f64(f).reshape(g.shape), _f64(a).reshape(g.shape), d, M, h, g)
    return g


def fidelity(geom: Geometry, f, y) -> float:
    return _load().ora_fidelity(geom.ref, _f64(f).reshape(geom.vol_shape), _f64(y).reshape(geom.proj_shape))


def reconstruct(geom: Geometry, y, f0, tau: float, d: int, M: int, h: float, mu: float, n_outer: int,
                n_inner: int = 1, clip: int = 1, gj_start: int = 0, with_report: bool = False, n_gj: int = 1,
                p1_cgls: int = 0):
    """TNLM-R (Sec. 2.3) with (P1) solved by n_inner gradient steps and (P2)
    by n_gj Eq. 8 iterations."""
    f = _f64(f0).reshape(geom.vol_shape).copy()
    rep = np.zeros((n_outer, n_inner), np.float64) if with_report else None
    _load().ora_reconstruct(geom.ref, _f64(y).reshape(geom.proj_shape), f, tau, d, M, h, mu, n_outer, n_inner,
                            n_gj, clip, gj_start, p1_cgls, rep.ctypes.data if rep is not None else None)
    return (f, rep) if with_report else f


def cgls(geom: Geometry, y, x0, n_iter: int, with_report: bool = False):
    """(P1) by CGLS phase by phase from x0; returns x (and the residual norms)."""
    x = _f64(x0).reshape(geom.vol_shape).copy()
    rep = np.zeros(n_iter + 1) if with_report else None
    _load().ora_cgls(geom.ref, _f64(y).reshape(geom.proj_shape), x, n_iter,
                     rep.ctypes.data if rep is not None else None)
    return (x, rep) if with_report else x


def fdk(geom: Geometry, proj, with_filtered: bool = False):
    """FDK of every phase from its own views (full-scan, ref. 16)."""
    out = np.empty(geom.vol_shape, np.float64)
    filt = np.empty(geom.proj_shape, np.float64) if with_filtered else None
    _load().ora_fdk(geom.ref, _f64(proj).reshape(geom.proj_shape), out,
                    filt.ctypes.data if filt is not None else None)
    return (out, filt) if with_filtered else out


def enhance(g, d: int, M: int, h: float, mu: float, n_sweeps: int, clip: int = 0) -> np.ndarray:
    """TNLM-E (Sec. 2.3): f^(0) = g, then n_sweeps weight+Eq. 8 sweeps."""
    g = _f64(g)
    np_, nz, ny, nx = g.shape
    f = np.empty_like(g)
    _load().ora_enhance(nx, ny, nz, np_, g, f, d, M, h, mu, n_sweeps, clip)
    return f


def num_threads() -> int:
    return _load().ora_num_threads()
