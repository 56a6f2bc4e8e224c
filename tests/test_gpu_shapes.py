"""Launch shapes and the autotuner: every compiled shape of the projector,
the band transpose and the box-sum sweep gives bit-identical outputs (same
operations in the same order per output), and tnlm_autotune picks a valid
shape without changing any result."""
import numpy as np
import pytest
import torch

import paper_1201_2450_gb300 as tnlm
from paper_1201_2450_gb300 import synth

pytestmark = pytest.mark.gpu

GEOMS = {
    "ragged_uneven": synth.make_geometry(nx=37, ny=29, nz=19, dx=1.0, nu=53, nv=27, du=1.3, sad=300, sdd=450,
                                         n_phases=3, views_per_phase=[4, 6, 5], angle_offset=0.13),
    "c1": synth.C1.geometry(),
}


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("name", list(GEOMS))
def test_projector_and_transpose_shapes_bitwise_equal(name):
    G = tnlm.Geometry(GEOMS[name])
    x = cuda(synth.uniform(G.vol_shape, 300))
    r = cuda(synth.uniform(G.proj_shape, 301))
    # a new handle starts at the table shape 104 and runs the slab walker until its tables exist
    assert tnlm.tnlm_get_launch_shapes(G)["projector_rows"] == 4
    tnlm.tnlm_project(G, x)
    assert tnlm.tnlm_get_launch_shapes(G)["projector_rows"] == 104
    outs_p, outs_b = [], []
    outs_t = []
    for rows in (2, 4, 8):  # the slab walker
        tnlm.tnlm_set_launch_shapes(G, rows, 8, 4)
        outs_p.append(tnlm.tnlm_project(G, x))
    for rows in (102, 104, 108):  # the table walker
        tnlm.tnlm_set_launch_shapes(G, rows, 8, 4)
        assert tnlm.tnlm_get_launch_shapes(G) == {"projector_rows": rows, "transpose_cells": 8, "transpose_rows": 4}
        outs_t.append(tnlm.tnlm_project(G, x))
    for cells in (4, 8):
        for rows in (2, 4):
            tnlm.tnlm_set_launch_shapes(G, 4, cells, rows)
            outs_b.append(tnlm.tnlm_backproject(G, r))
    torch.cuda.synchronize()
    for o in outs_p[1:]:
        assert torch.equal(o, outs_p[0])
    for o in outs_t[1:]:
        assert torch.equal(o, outs_t[0])
    # the two walkers agree to FP32 rounding
    d = (outs_t[0].double() - outs_p[0].double()).norm() / outs_p[0].double().norm()
    assert float(d) <= 1e-6
    for o in outs_b[1:]:
        assert torch.equal(o, outs_b[0])


@pytest.mark.parametrize("name", list(GEOMS))
def test_projector_shapes_residual_path_bitwise_equal(name):
    """The fused residual (FP32 and BF16 storage) through one TNLM-R iteration:
    the same image for every projector shape of one walker."""
    G = tnlm.Geometry(GEOMS[name])
    y = cuda(synth.uniform(G.proj_shape, 302) * 0.3)
    f0 = cuda(synth.smooth_volume(G.vol_shape, 303))
    p = tnlm.Params(d=1, M=2, h=0.02, mu=0.8, tau=1e-4, n_outer=1)
    for family in ((2, 4, 8), (102, 104, 108)):
        outs, outs16 = [], []
        for rows in family:
            tnlm.tnlm_set_launch_shapes(G, rows, 8, 4)
            f = f0.clone()
            tnlm.tnlm_reconstruct(G, y, f, p)
            outs.append(f)
            f16 = f0.bfloat16()
            tnlm.tnlm_reconstruct_bf16(G, y.bfloat16(), f16, p)
            outs16.append(f16)
        torch.cuda.synchronize()
        for o in outs[1:]:
            assert torch.equal(o, outs[0])
        for o in outs16[1:]:
            assert torch.equal(o, outs16[0])


@pytest.mark.parametrize("d, M", [(1, 1), (1, 2), (1, 3), (2, 1), (2, 2), (2, 3)])
def test_sweep_shapes_bitwise_equal(d, M):
    shape = (3, 21, 27, 35)  # ragged against every tile
    a = cuda(synth.smooth_volume(shape, 310) + synth.normal(shape, 311, 0.01))
    g = cuda(synth.smooth_volume(shape, 312))
    outs, outs16 = [], []
    try:
        for s in range(4):
            tnlm.tnlm_set_sweep_shape(d, M, False, s)
            tnlm.tnlm_set_sweep_shape(d, M, True, s)
            outs.append(tnlm.tnlm_gauss_jacobi(a, a, g, d, M, 0.05, 1.0, clip=1))
            outs16.append(tnlm.tnlm_gauss_jacobi_bf16(a.bfloat16(), a.bfloat16(), g.bfloat16(), d, M, 0.05, 1.0, clip=1))
        torch.cuda.synchronize()
    finally:
        tnlm.tnlm_set_sweep_shape(d, M, False, 0)
        tnlm.tnlm_set_sweep_shape(d, M, True, 0)
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    for o in outs16[1:]:
        assert torch.equal(o, outs16[0])


def test_autotune_keeps_results():
    G = tnlm.Geometry(GEOMS["ragged_uneven"])
    y = cuda(synth.uniform(G.proj_shape, 320) * 0.3)
    f0 = synth.smooth_volume(G.vol_shape, 321)
    p = tnlm.Params(d=1, M=2, h=0.02, mu=0.8, tau=1e-4, n_outer=2)
    before = cuda(f0)
    tnlm.tnlm_reconstruct(G, y, before, p)
    try:
        ch = tnlm.tnlm_autotune(G, p)
        assert ch["projector_rows"] in (102, 104, 108)
        assert ch["transpose_cells"] in (4, 8) and ch["transpose_rows"] in (2, 4)
        assert 0 <= ch["sweep_shape"] < 4
        after = cuda(f0)
        tnlm.tnlm_reconstruct(G, y, after, p)
        torch.cuda.synchronize()
        assert torch.equal(before, after)
        s = tnlm.tnlm_autotune_sweep((3, 16, 20, 24), 2, 3, 0.04, bf16=True)
        assert 0 <= s < 4
    finally:
        tnlm.tnlm_set_sweep_shape(1, 2, False, 0)
        tnlm.tnlm_set_sweep_shape(2, 3, True, 0)
