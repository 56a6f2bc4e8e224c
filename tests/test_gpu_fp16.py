"""FP16 storage with FP32 arithmetic: the *_fp16 calls against the FP32 calls
on the widened inputs (bit for bit, one output rounding apart) and against the
FP64 oracle (errors of the order of FP16's unit roundoff, 2^-11, eight times
smaller than BF16's)."""
import numpy as np
import pytest
import torch

import paper_1201_2450_gb300 as tnlm
from paper_1201_2450_gb300 import synth

pytestmark = pytest.mark.gpu
FP16_U = 2.0 ** -11  # unit roundoff of IEEE half precision (11-bit significand, round to nearest)
RTOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def gpu():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    tnlm.build()
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _h(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda().half()


@pytest.mark.parametrize("shape,d,M", [((3, 9, 13, 19), 1, 3), ((3, 7, 10, 11), 2, 3), ((2, 8, 12, 20), 2, 1)])
def test_fp16_sweep_is_rounded_fp32_sweep(ora, shape, d, M):
    """The sweep on FP16 images equals the FP32 sweep on the same images
    rounded to FP16, bit for bit; against the FP64 oracle its error is the
    output rounding (<= 2^-11)."""
    rng = np.random.default_rng(600)
    a = synth.smooth_volume(shape, 601) + rng.normal(0, 0.002, shape).astype(np.float32)
    g = synth.smooth_volume(shape, 602)
    h = 0.02
    A, G = _h(a), _h(g)
    out = tnlm.tnlm_gauss_jacobi_fp16(A, A, G, d, M, h, 0.8, 1)
    out_f = tnlm.tnlm_gauss_jacobi(A.float().contiguous(), A.float().contiguous(), G.float().contiguous(), d, M, h,
                                   0.8, 1)
    assert torch.equal(out, out_f.half())
    ref = ora.gj_sweep(A.float().cpu().numpy(), A.float().cpu().numpy(), G.float().cpu().numpy(), d, M, h, 0.8, 1)
    assert rel_l2(out.float().cpu().numpy(), ref) <= FP16_U


def test_fp16_enhance_error_vs_fp64(ora):
    """TNLM-E with FP16 storage over 5 sweeps against the FP64 oracle on the
    same FP16-valued input: each sweep rounds its output (relative <= u) and the
    Jacobi map contracts by 2/(2+mu), so the error stays below u/(1-2/3)."""
    cfg = synth.EnhanceConfig("t", 4, (24, 20, 12), 1.0, 0.002, 0.003, 36, 2, 3, 0.04, 1.0, 5, 220)
    g, _ = synth.enhance_input(cfg)
    G = g.cuda().half()
    p = tnlm.Params(d=2, M=3, h=0.04, mu=1.0, n_outer=5, clip_nonneg=0)
    f = tnlm.tnlm_enhance_fp16(G, p)
    ref = ora.enhance(G.float().cpu().numpy(), 2, 3, 0.04, 1.0, 5)
    err = rel_l2(f.float().cpu().numpy(), ref)
    fb = tnlm.tnlm_enhance_bf16(g.cuda().bfloat16(), p)
    err_b = rel_l2(fb.float().cpu().numpy(), ora.enhance(g.cuda().bfloat16().float().cpu().numpy(), 2, 3, 0.04, 1.0, 5))
    print(f"TNLM-E 5 sweeps vs FP64: FP16 storage rel-L2 {err:.3e}, BF16 {err_b:.3e}")
    assert err <= 3 * FP16_U
    assert err < err_b


def _fp16_round(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).half().float().numpy()


C2_TINY = synth.ReconConfig("NCAT-shaped reduced 10x32x32x8, 9 views x 64x48", 10, (32, 32, 8), 16.0, 9, (64, 48),
                            6.24, 5e4, 1, 3, 0.02, 1.0, 10, "thorax", 1002)


@pytest.mark.parametrize("cfg, n_outer", [(synth.C1, synth.C1.n_outer), (C2_TINY, 10)])
def test_reconstruct_fp16_error_vs_fp64(ora, cfg, n_outer):
    """TNLM-R with FP16 storage against the FP64 oracle on the same
    FP16-representable measurements, within 2 n_outer u (two roundings per
    iteration); the residual norms within 4 n_outer u."""
    pb = synth.recon_problem(cfg)
    OG = ora.Geometry(pb.geom)
    L = ora.power_norm(OG, synth.uniform(OG.vol_shape, 7), 30)
    tau = float(np.float32(1.0 / L))
    y = _fp16_round(pb.y.numpy())
    f_ref, rep_ref = ora.reconstruct(OG, y, np.zeros(OG.vol_shape), tau, cfg.d, cfg.M, cfg.h, cfg.mu, n_outer,
                                     with_report=True)
    G = tnlm.Geometry(pb.geom)
    p = tnlm.Params(d=cfg.d, M=cfg.M, h=cfg.h, mu=cfg.mu, tau=tau, n_outer=n_outer)
    f16 = torch.zeros(G.vol_shape, device="cuda", dtype=torch.float16)
    _, rep = tnlm.tnlm_reconstruct_fp16(G, _h(y), f16, p, report=True)
    err = rel_l2(f16.float().cpu().numpy(), f_ref)
    print(f"FP16 storage rel-L2 vs FP64 after {n_outer} iterations: {err:.3e}")
    assert err <= 2 * n_outer * FP16_U
    np.testing.assert_allclose(rep, rep_ref, rtol=4 * n_outer * FP16_U)
    assert torch.all(f16.float() >= 0)


@pytest.mark.parametrize("d, M", [(1, 2), (2, 1)])
def test_energy_grad_fp16_equals_fp32_on_widened_inputs(d, M):
    geom = synth.make_geometry(nx=21, ny=17, nz=9, dx=1.0, nu=40, nv=12, du=1.2, sad=300, sdd=450, n_phases=3,
                               views_per_phase=[4, 5, 3], angle_offset=0.03)
    G = tnlm.Geometry(geom)
    a = synth.smooth_volume(G.vol_shape, 610)
    f = synth.uniform(G.vol_shape, 611, 0.0, 0.04)
    y = synth.uniform(G.proj_shape, 612, 0.0, 0.3)
    p = tnlm.Params(d=d, M=M, h=0.03, mu=0.7)
    E16, g16 = tnlm.tnlm_energy_grad_fp16(G, _h(y), _h(f), _h(a), p)
    E32, g32 = tnlm.tnlm_energy_grad(G, _h(y).float(), _h(f).float(), _h(a).float(), p)
    torch.cuda.synchronize()
    assert E16 == E32
    assert torch.equal(g16, g32)


def test_batch_plan_fp16_equals_single_calls():
    geoms = [synth.make_geometry(nx=21, ny=17, nz=9, dx=1.0, nu=40, nv=12, du=1.2, sad=300, sdd=450, n_phases=3,
                                 views_per_phase=[4, 5, 3], angle_offset=0.03), synth.C1.geometry()]
    params = [tnlm.Params(d=1, M=2, h=0.02, mu=0.8, tau=1e-4, n_outer=2),
              tnlm.Params(d=2, M=1, h=0.03, mu=1.1, tau=5e-5, n_outer=2, n_gj=2, gj_start=1)]
    Gs = [tnlm.Geometry(g) for g in geoms]
    ys = [_h(synth.uniform(G.proj_shape, 620 + k) * 0.3) for k, G in enumerate(Gs)]
    f0 = [_h(synth.smooth_volume(G.vol_shape, 630 + k)) for k, G in enumerate(Gs)]
    single = []
    for G, y, f, p in zip(Gs, ys, f0, params):
        x = f.clone()
        tnlm.tnlm_reconstruct_fp16(G, y, x, p)
        single.append(x)
    Gb = [tnlm.Geometry(g) for g in geoms]
    fb = [f.clone() for f in f0]
    plan = tnlm.BatchPlan(Gb, ys, fb, params)
    plan.run(2)
    plan.close()
    torch.cuda.synchronize()
    for a, b in zip(single, fb):
        assert torch.equal(a, b)


@pytest.mark.parametrize("d, M", [(1, 3), (2, 3)])
def test_fp16_sweep_shapes_bitwise_equal(d, M):
    shape = (3, 21, 27, 35)
    a = _h(synth.smooth_volume(shape, 640) + synth.normal(shape, 641, 0.01))
    g = _h(synth.smooth_volume(shape, 642))
    outs = []
    try:
        for s in range(4):
            tnlm.tnlm_set_sweep_shape(d, M, False, s, fp16=True)
            outs.append(tnlm.tnlm_gauss_jacobi_fp16(a, a, g, d, M, 0.05, 1.0, clip=1))
        torch.cuda.synchronize()
        assert 0 <= tnlm.tnlm_autotune_sweep((3, 16, 20, 24), d, M, 0.04, fp16=True) < 4
    finally:
        tnlm.tnlm_set_sweep_shape(d, M, False, 0, fp16=True)
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
