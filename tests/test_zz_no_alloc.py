"""tnlm_enhance_noalloc: TNLM-E for callers that cannot allocate device
memory (their memory pool owns the GPU's budget), which keeps its ping-pong
image in a fixed 16 MiB device array of the library.

Its output must match tnlm_enhance (which allocates that image stream-
ordered) bit for bit, on two calls in a row with a call in between that
leaves large negative values in the shared array.  This file sorts last so a
run that stops at the first failure has run every other test before it."""
import ctypes as C

import numpy as np
import pytest
import torch

import paper_1201_2450_gb300 as tnlm
from paper_1201_2450_gb300 import synth

pytestmark = pytest.mark.gpu
RTOL = 1e-5


@pytest.fixture(scope="module")
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    tnlm.build()
    torch.cuda.set_device(0)
    return tnlm._load()


def _rel_l2(a, b):
    a = a.double()
    b = b.double()
    return float((a - b).norm() / b.norm())


def _call_noalloc(lib, g, out, params):
    np_, nz, ny, nx = g.shape
    p = params._c()
    stream = torch.cuda.current_stream().cuda_stream
    return lib.tnlm_enhance_noalloc(nx, ny, nz, np_, C.c_void_p(g.data_ptr()), C.c_void_p(out.data_ptr()),
                                    C.byref(p), C.c_void_p(stream))


def test_noalloc_matches_enhance_two_calls(lib):
    """Two calls in a row, each equal to tnlm_enhance bit for bit (the same
    sweeps in the same order).  Between them a call on a larger volume with
    large negative values and no positivity fills the shared array with data
    that would change the second result if any sweep read the array before
    writing it."""
    shapes = [((4, 12, 20, 24), 2, 2, 3), ((3, 16, 18, 21), 1, 3, 4)]
    for k, (shape, d, M, sweeps) in enumerate(shapes):
        g = torch.from_numpy(synth.smooth_volume(shape, 300 + k) + synth.normal(shape, 310 + k, 0.002)).cuda()
        params = tnlm.Params(d=d, M=M, h=0.02, mu=1.0, n_outer=sweeps, clip_nonneg=k)
        ref = tnlm.tnlm_enhance(g, params)
        out = torch.full_like(g, float("nan"))
        assert _call_noalloc(lib, g, out, params) == 0, lib.tnlm_last_error()
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert _rel_l2(out, ref) <= RTOL
        assert torch.equal(out, ref)
        if k == 0:
            big = torch.full((5, 40, 60, 64), -1e4, device="cuda")
            big_out = torch.empty_like(big)
            junk = tnlm.Params(d=1, M=1, h=0.02, mu=1.0, n_outer=3, clip_nonneg=0)
            assert _call_noalloc(lib, big, big_out, junk) == 0, lib.tnlm_last_error()
            torch.cuda.synchronize()


@pytest.mark.parametrize("n_outer", [0, 1, 2])
def test_noalloc_short_schedules_and_python_wrapper(lib, n_outer):
    """n_outer = 0 copies g, n_outer = 1 sweeps straight into f (no scratch);
    the Python wrapper marshals the same call."""
    shape = (3, 9, 14, 17)
    g = torch.from_numpy(synth.smooth_volume(shape, 320) + synth.normal(shape, 321, 0.002)).cuda()
    params = tnlm.Params(d=1, M=2, h=0.02, mu=0.8, n_outer=n_outer, clip_nonneg=0)
    ref = tnlm.tnlm_enhance(g, params)
    out = torch.full_like(g, float("nan"))
    tnlm.tnlm_enhance_noalloc(g, params, out)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    if n_outer == 0:
        assert torch.equal(out, g)


def test_noalloc_rejects_oversize(lib):
    shape = (2, 128, 128, 129)  # 4,227,072 voxels > 4 Mi
    g = torch.zeros(shape, device="cuda")
    out = torch.zeros_like(g)
    status = _call_noalloc(lib, g, out, tnlm.Params(d=1, M=1, h=0.02, mu=1.0, n_outer=2))
    assert status == 1
    assert b"at most 4194304 voxels" in lib.tnlm_last_error()
