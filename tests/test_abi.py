"""The C-ABI library builds for sm_103a, loads, exports every function that
include/tnlm.h declares, and rejects invalid arguments on the host before any
CUDA call (these checks need no GPU)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_1201_2450_gb300 as tnlm
from paper_1201_2450_gb300 import synth

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "tnlm.h")


@pytest.fixture(scope="module")
def lib():
    tnlm.build()
    return tnlm._load()


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tnlm_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("tnlm_create_geometry", "tnlm_project", "tnlm_backproject", "tnlm_weights",
                     "tnlm_gauss_jacobi", "tnlm_reconstruct", "tnlm_enhance"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    assert lib.tnlm_status_string(0) == b"ok"
    assert lib.tnlm_status_string(1) == b"invalid argument"
    assert lib.tnlm_version() >= 10000


def _desc(**over):
    g = synth.make_geometry(nx=8, ny=8, nz=4, dx=1.0, nu=16, nv=8, du=1.5, n_phases=2, views_per_phase=3)
    g.update(over)
    return g


@pytest.mark.parametrize("over, msg", [
    (dict(nx=0), "volume dimensions"),
    (dict(dx=-1.0), "voxel sizes"),
    (dict(sdd=900.0), "sad < sdd"),
    (dict(nviews=np.array([], np.int32), angles=np.zeros(0)), "n_phases"),
    (dict(nviews=np.array([3, 0], np.int32), angles=np.zeros(3)), "at least one view"),
    (dict(nx=2000, dx=1.0), "inside the source circle"),
    (dict(nv=7000), "nv must not exceed"),
])
def test_create_geometry_rejects(lib, over, msg):
    with pytest.raises(tnlm.TnlmError) as e:
        tnlm.Geometry(_desc(**over))
    assert e.value.status == 1
    assert msg in str(e.value)


def test_sweep_argument_checks(lib):
    vp = C.c_void_p(16)
    # N_p = 1 is rejected (it would compare a phase with itself)
    assert lib.tnlm_gauss_jacobi(4, 4, 4, 1, vp, vp, vp, C.c_void_p(32), 1, 1, 0.1, 1.0, 0, None) == 1
    assert b"n_phases" in lib.tnlm_last_error()
    assert lib.tnlm_gauss_jacobi(4, 4, 4, 2, vp, vp, vp, C.c_void_p(32), 1, 9, 0.1, 1.0, 0, None) == 1
    assert lib.tnlm_gauss_jacobi(4, 4, 4, 2, vp, vp, vp, C.c_void_p(32), 1, 1, 0.0, 1.0, 0, None) == 1
    assert lib.tnlm_gauss_jacobi(4, 4, 4, 2, vp, vp, vp, vp, 1, 1, 0.1, 1.0, 0, None) == 1  # aliasing
    assert b"alias" in lib.tnlm_last_error()
    # the range sweep: output phases must lie inside the arrays' phases
    assert lib.tnlm_gauss_jacobi_range(4, 4, 4, 3, 1, 3, vp, vp, vp, C.c_void_p(32), 1, 1, 0.1, 1.0, 0, None) == 1
    assert b"must lie inside" in lib.tnlm_last_error()
    assert lib.tnlm_gauss_jacobi_range(4, 4, 4, 3, -1, 1, vp, vp, vp, C.c_void_p(32), 1, 1, 0.1, 1.0, 0, None) == 1
    assert lib.tnlm_gauss_jacobi_range(4, 4, 4, 3, 1, 1, vp, vp, vp, vp, 1, 1, 0.1, 1.0, 0, None) == 1  # aliasing
    assert b"alias" in lib.tnlm_last_error()
    # (P1) alone: null and aliased arguments are rejected before any device work
    assert lib.tnlm_p1(None, vp, vp, C.c_void_p(32), None, None, None) == 1
    assert lib.tnlm_p1(vp, vp, vp, vp, None, None, None) == 1
    # weight buffer too small
    assert lib.tnlm_weights(4, 4, 4, 2, vp, 1, 1, 0.1, vp, 10, None) == 1
    assert b"needed" in lib.tnlm_last_error()


def test_batch_plan_rejects_bad_arguments(lib):
    lib = C.CDLL(tnlm.library_path())  # own function objects: the binding's argtypes stay untouched
    lib.tnlm_last_error.restype = C.c_char_p
    lib.tnlm_batch_plan_create.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.POINTER(C.c_void_p)]
    out = C.c_void_p(1)
    assert lib.tnlm_batch_plan_create(0, None, None, None, None, C.byref(out)) == 1
    assert out.value is None
    assert b"n >= 1" in lib.tnlm_last_error()
    lib.tnlm_batch_plan_run.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
    assert lib.tnlm_batch_plan_run(None, 1, None) == 1
    lib.tnlm_batch_plan_destroy.argtypes = [C.c_void_p]
    lib.tnlm_batch_plan_destroy(None)  # NULL is ignored


def test_launch_shape_setters_reject_uncompiled_shapes(lib):
    lib = C.CDLL(tnlm.library_path())
    lib.tnlm_last_error.restype = C.c_char_p
    assert lib.tnlm_set_sweep_shape(1, 3, 0, 4) == 1
    assert b"shape" in lib.tnlm_last_error()
    assert lib.tnlm_set_sweep_shape(5, 3, 0, 0) == 1
    lib.tnlm_set_launch_shapes.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int]
    assert lib.tnlm_set_launch_shapes(None, 4, 8, 4) == 1
    lib.tnlm_reconstruct_host.argtypes = [C.c_void_p] * 8
    assert lib.tnlm_reconstruct_host(None, None, None, None, None, None, None, None) == 1
    assert b"must not be NULL" in lib.tnlm_last_error()
    lib.tnlm_get_launch_shapes.argtypes = [C.c_void_p, C.c_void_p]
    out = (C.c_int * 3)()
    assert lib.tnlm_get_launch_shapes(None, out) == 1
