"""GPU parity: every C-ABI call against the FP64 oracle on seeded inputs.

Tolerance: relative L2 error <= 1e-5 for the FP32 paths (elementwise
comparison over the whole output), as the method's FP32 target states.
Sizes span several CUDA tiles with ragged tails (projector tiles 32 x 4
pixels, transpose tiles 32 x 4 columns x 8 slices, sweep tiles 8 x 8 x 4).
At the full benchmark size (10 x 256^2 x 64, 36 views x 512 x 384) outputs
are checked on sampled rays / voxels the oracle computes one by one and via
the adjoint identity, which holds at any size."""
import math

import numpy as np
import pytest
import torch

import paper_1201_2450_gb300 as tnlm
from paper_1201_2450_gb300 import synth

pytestmark = pytest.mark.gpu
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


def cuda(x):
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float32)).cuda()


GEOMS = {
    "ragged_uneven": synth.make_geometry(nx=37, ny=29, nz=11, dx=1.0, dy=1.1, dz=0.9, cx=0.7, cy=-1.3, cz=0.4,
                                         nu=70, nv=13, du=1.3, dv=1.7, u_off=0.9, v_off=-0.6, sad=300.0,
                                         sdd=450.0, n_phases=3, views_per_phase=[4, 5, 3], angle_offset=0.03),
    "c1": synth.C1.geometry(),
}


@pytest.mark.parametrize("name", list(GEOMS))
def test_project_matches_oracle(ora, name):
    geom = GEOMS[name]
    G = tnlm.Geometry(geom)
    OG = ora.Geometry(geom)
    x = synth.uniform(G.vol_shape, 101)
    p = tnlm.tnlm_project(G, cuda(x)).cpu().numpy()
    p_ref = ora.project(OG, x)
    assert rel_l2(p, p_ref) <= RTOL


@pytest.mark.parametrize("name", list(GEOMS))
def test_backproject_matches_oracle(ora, name):
    geom = GEOMS[name]
    G = tnlm.Geometry(geom)
    OG = ora.Geometry(geom)
    y = synth.uniform(G.proj_shape, 102)
    v0 = synth.uniform(G.vol_shape, 103)
    out = tnlm.tnlm_backproject(G, cuda(y), cuda(v0), alpha=2.0, beta=0.5).cpu().numpy()
    ref = 0.5 * v0.astype(np.float64) + 2.0 * ora.backproject(OG, y)
    assert rel_l2(out, ref) <= RTOL
    bt = tnlm.tnlm_backproject(G, cuda(y)).cpu().numpy()
    assert rel_l2(bt, ora.backproject(OG, y)) <= RTOL


def test_tall_detector_pair_matches_oracle(ora):
    """A 4096-row detector: the per-row table of the transpose (16 B per row)
    needs more than the default 48 KB of shared memory; projector and
    transpose still match the oracle."""
    geom = synth.make_geometry(nx=12, ny=11, nz=10, dx=1.0, nu=16, nv=4096, du=1.0, dv=0.01, sad=300.0, sdd=450.0,
                               n_phases=2, views_per_phase=[3, 4], angle_offset=0.2)
    G = tnlm.Geometry(geom)
    OG = ora.Geometry(geom)
    x = synth.uniform(G.vol_shape, 104)
    assert rel_l2(tnlm.tnlm_project(G, cuda(x)).cpu().numpy(), ora.project(OG, x)) <= RTOL
    y = synth.uniform(G.proj_shape, 105)
    assert rel_l2(tnlm.tnlm_backproject(G, cuda(y)).cpu().numpy(), ora.backproject(OG, y)) <= RTOL


@pytest.mark.parametrize("name", list(GEOMS))
def test_adjoint_identity_gpu_pair(name):
    G = tnlm.Geometry(GEOMS[name])
    x = cuda(synth.uniform(G.vol_shape, 104))
    y = cuda(synth.uniform(G.proj_shape, 105))
    px = tnlm.tnlm_project(G, x)
    bty = tnlm.tnlm_backproject(G, y)
    lhs = float((px.double() * y.double()).sum())
    rhs = float((x.double() * bty.double()).sum())
    assert abs(lhs - rhs) <= 1e-6 * float(px.double().norm() * y.double().norm())


def test_project_odd_detector_face_rays(ora):
    """Odd nu, nv put pixel rays exactly in voxel face planes at multiples of
    90 degrees; away from such exact ties the pair still matches."""
    geom = synth.make_geometry(nx=16, ny=16, nz=8, dx=1.0, nu=33, nv=17, du=1.0, sad=200, sdd=300, n_phases=2,
                               views_per_phase=3, angle_offset=0.01)
    G = tnlm.Geometry(geom)
    x = synth.uniform(G.vol_shape, 106)
    assert rel_l2(tnlm.tnlm_project(G, cuda(x)).cpu().numpy(), ora.project(ora.Geometry(geom), x)) <= RTOL


def test_backproject_thin_slices_fallback(ora):
    """Thin slices and a tall detector: a chord can span several z cells, so the
    library takes its exact per-cell transpose instead of the band/prefix-sum
    one; both must match the oracle."""
    geom = synth.make_geometry(nx=12, ny=10, nz=20, dx=1.0, dz=0.15, nu=40, nv=64, du=1.0, dv=2.0, sad=150.0,
                               sdd=300.0, n_phases=2, views_per_phase=[3, 4], angle_offset=0.2)
    G = tnlm.Geometry(geom)
    y = synth.uniform(G.proj_shape, 108)
    out = tnlm.tnlm_backproject(G, cuda(y)).cpu().numpy()
    assert rel_l2(out, ora.backproject(ora.Geometry(geom), y)) <= RTOL
    x = cuda(synth.uniform(G.vol_shape, 109))
    px = tnlm.tnlm_project(G, x)
    bty = tnlm.tnlm_backproject(G, cuda(y))
    lhs = float((px.double() * cuda(y).double()).sum())
    rhs = float((x.double() * bty.double()).sum())
    assert abs(lhs - rhs) <= 1e-6 * float(px.double().norm() * cuda(y).double().norm())


WEIGHT_CASES = [((3, 7, 10, 12), 1, 2, 0.5), ((2, 5, 6, 9), 2, 1, 0.8), ((4, 4, 4, 4), 0, 2, 0.3),
                ((2, 6, 5, 7), 1, 3, 0.5)]


@pytest.mark.parametrize("shape,d,M,h", WEIGHT_CASES)
def test_weights_match_oracle(ora, shape, d, M, h):
    a = synth.uniform(shape, 107)
    w = tnlm.tnlm_weights(cuda(a), d, M, h).cpu().numpy()
    ref = ora.weights(a, d, M, h)
    assert rel_l2(w, ref) <= RTOL
    np.testing.assert_allclose(w.sum(-1), 1.0, rtol=1e-5)


def test_weights_hand_fixture():
    """The 2-phase 4^3 fixture of tests/golden (hand-derived closed forms)."""
    a = np.zeros((2, 4, 4, 4), np.float32)
    a[0, 1, 1, 1] = 1.0
    a[1, 1, 1, 2] = 1.0
    w = tnlm.tnlm_weights(cuda(a), 1, 1, 1.0).cpu().numpy()
    assert w[0, 0, 1, 1, 1][14] == pytest.approx(1.0 / (1 + 9 * math.exp(-0.5) + 17 * math.exp(-1)), rel=1e-6)
    assert w[0, 0, 0, 0, 0][14] == pytest.approx(1.0 / (1 + 4 * math.exp(-0.5) + 3 * math.exp(-1)), rel=1e-6)


def _sweep_inputs(shape, seed, kind):
    if kind == "smooth":
        a = synth.smooth_volume(shape, seed) + synth.normal(shape, seed + 1, 0.002)
        v = a + synth.normal(shape, seed + 2, 0.001)
        g = a + synth.normal(shape, seed + 3, 0.003)
        return a, v, g, 0.02
    a = synth.uniform(shape, seed)
    return a, synth.uniform(shape, seed + 1), synth.uniform(shape, seed + 2) - 0.3, 0.6


SWEEP_CASES = [
    ((3, 9, 13, 19), 1, 1, "smooth", 0), ((2, 9, 13, 19), 1, 2, "uniform", 1), ((4, 9, 13, 19), 1, 3, "smooth", 1),
    ((3, 7, 10, 11), 2, 3, "smooth", 0), ((3, 7, 10, 11), 2, 2, "uniform", 0), ((2, 5, 9, 8), 0, 2, "uniform", 0),
    ((3, 6, 9, 10), 3, 1, "smooth", 1), ((5, 4, 8, 8), 1, 0, "uniform", 0), ((3, 9, 17, 33), 2, 1, "smooth", 1),
]


@pytest.mark.parametrize("shape,d,M,kind,clip", SWEEP_CASES)
def test_gauss_jacobi_matches_oracle(ora, shape, d, M, kind, clip):
    a, v, g, h = _sweep_inputs(shape, 110, kind)
    mu = 0.8
    out = tnlm.tnlm_gauss_jacobi(cuda(a), cuda(v), cuda(g), d, M, h, mu, clip).cpu().numpy()
    ref = ora.gj_sweep(a, v, g, d, M, h, mu, clip)
    assert rel_l2(out, ref) <= RTOL


def test_gauss_jacobi_window_zero_closed_form():
    """M = 0: the window is the voxel itself, so Eq. 8 reduces to
    (mu g_i + v_{i+1} + v_{i-1}) / (2 + mu) whatever the weights."""
    shape = (3, 5, 6, 7)
    a, v, g = (synth.uniform(shape, s) for s in (120, 121, 122))
    out = tnlm.tnlm_gauss_jacobi(cuda(a), cuda(v), cuda(g), 1, 0, 0.1, 0.5).cpu().numpy()
    ref = (0.5 * g + np.roll(v, -1, 0) + np.roll(v, 1, 0)) / 2.5
    np.testing.assert_allclose(out, ref, rtol=2e-6, atol=1e-7)


def test_gauss_jacobi_single_voxel_volume():
    shape = (2, 1, 1, 1)
    a, v, g = (synth.uniform(shape, s) for s in (123, 124, 125))
    out = tnlm.tnlm_gauss_jacobi(cuda(a), cuda(v), cuda(g), 2, 3, 0.1, 1.0).cpu().numpy()
    ref = (g + 2 * v[::-1]) / 3.0
    np.testing.assert_allclose(out, ref, rtol=2e-6)


def test_enhance_matches_oracle(ora):
    shape = (4, 12, 20, 24)
    cfg = synth.EnhanceConfig("t", 4, (24, 20, 12), 1.0, 0.002, 0.003, 36, 2, 3, 0.04, 1.0, 3, 130)
    g, _ = synth.enhance_input(cfg)
    g = g.numpy()
    p = tnlm.Params(d=2, M=3, h=0.04, mu=1.0, n_outer=3, clip_nonneg=0)
    f = tnlm.tnlm_enhance(cuda(g), p).cpu().numpy()
    ref = ora.enhance(g, 2, 3, 0.04, 1.0, 3)
    assert rel_l2(f, ref) <= RTOL
    # zero sweeps copy g; two sweeps end in the output buffer too
    p0 = tnlm.Params(d=2, M=3, h=0.04, mu=1.0, n_outer=0, clip_nonneg=0)
    np.testing.assert_array_equal(tnlm.tnlm_enhance(cuda(g), p0).cpu().numpy(), g)
    p2 = tnlm.Params(d=1, M=2, h=0.04, mu=1.0, n_outer=2, clip_nonneg=0)
    assert rel_l2(tnlm.tnlm_enhance(cuda(g), p2).cpu().numpy(), ora.enhance(g, 1, 2, 0.04, 1.0, 2)) <= RTOL


C3_TINY = synth.EnhanceConfig("TNLM-E reduced 10x20x20x8", 10, (20, 20, 8), 9.6, 0.002, 0.003, 36, 2, 3, 0.04, 1.0, 30,
                              1003)


def test_enhance_c3_structure_full_length(ora):
    """C3's structure (10 phases, patch 5^3, window 7^3, h = 0.04) for its full 30 sweeps on a reduced grid."""
    cfg = C3_TINY
    g, _ = synth.enhance_input(cfg)
    g = g.numpy()
    p = tnlm.Params(d=cfg.d, M=cfg.M, h=cfg.h, mu=cfg.mu, n_outer=cfg.n_sweeps, clip_nonneg=0)
    f = tnlm.tnlm_enhance(cuda(g), p).cpu().numpy()
    ref = ora.enhance(g, cfg.d, cfg.M, cfg.h, cfg.mu, cfg.n_sweeps)
    assert rel_l2(f, ref) <= RTOL


def _recon_case(ora, cfg, n_outer, seed=7):
    pb = synth.recon_problem(cfg)
    OG = ora.Geometry(pb.geom)
    L = ora.power_norm(OG, synth.uniform(OG.vol_shape, seed), 30)
    tau = float(np.float32(1.0 / L))
    y = pb.y.numpy()
    f_ref, rep_ref = ora.reconstruct(OG, y, np.zeros(OG.vol_shape), tau, cfg.d, cfg.M, cfg.h, cfg.mu, n_outer,
                                     with_report=True)
    G = tnlm.Geometry(pb.geom)
    f = torch.zeros(G.vol_shape, device="cuda")
    p = tnlm.Params(d=cfg.d, M=cfg.M, h=cfg.h, mu=cfg.mu, tau=tau, n_outer=n_outer)
    _, rep = tnlm.tnlm_reconstruct(G, cuda(y), f, p, report=True)
    return f.cpu().numpy(), f_ref, rep, rep_ref


def test_reconstruct_c1_full(ora):
    """Config C1 in full: 4 x 32^3, 20 views x 64 x 48, d=1, M=2, 5 iterations."""
    f, f_ref, rep, rep_ref = _recon_case(ora, synth.C1, synth.C1.n_outer)
    assert rel_l2(f, f_ref) <= RTOL
    np.testing.assert_allclose(rep, rep_ref, rtol=RTOL)
    assert np.all(f >= 0)


C2_TINY = synth.ReconConfig("NCAT-shaped reduced 10x32x32x8, 9 views x 64x48", 10, (32, 32, 8), 16.0, 9, (64, 48),
                            6.24, 5e4, 1, 3, 0.02, 1.0, 50, "thorax", 1002)


def test_reconstruct_c2_structure_full_length(ora):
    """C2's structure (10 phases, d=1, M=3, 50 FBS iterations) at a reduced grid."""
    f, f_ref, rep, rep_ref = _recon_case(ora, C2_TINY, C2_TINY.n_outer)
    err = rel_l2(f, f_ref)
    assert err <= RTOL, err
    np.testing.assert_allclose(rep, rep_ref, rtol=RTOL)


def test_reconstruct_gj_start_and_inner_steps(ora):
    geom = GEOMS["ragged_uneven"]
    OG = ora.Geometry(geom)
    G = tnlm.Geometry(geom)
    y = synth.uniform(G.proj_shape, 140) * 0.5
    f0 = synth.smooth_volume(G.vol_shape, 141)
    tau = 1e-4
    ref = ora.reconstruct(OG, y, f0, tau, 1, 2, 0.02, 0.7, 2, n_inner=3, clip=0, gj_start=1)
    f = cuda(f0)
    tnlm.tnlm_reconstruct(G, cuda(y), f, tnlm.Params(d=1, M=2, h=0.02, mu=0.7, tau=tau, n_outer=2, n_inner=3,
                                                     clip_nonneg=0, gj_start=1))
    assert rel_l2(f.cpu().numpy(), ref) <= RTOL
    # n_outer = 0 leaves f untouched
    f = cuda(f0)
    tnlm.tnlm_reconstruct(G, cuda(y), f, tnlm.Params(tau=tau, n_outer=0))
    np.testing.assert_array_equal(f.cpu().numpy(), f0)


def test_operator_norm_matches_oracle(ora):
    geom = GEOMS["ragged_uneven"]
    x0 = synth.uniform((3, 11, 29, 37), 150)
    L_ref = ora.power_norm(ora.Geometry(geom), x0, 40)
    G = tnlm.Geometry(geom)
    L = tnlm.tnlm_operator_norm(G, cuda(x0), 40)
    assert L == pytest.approx(L_ref, rel=1e-4)


def test_stage_timing_counts_launches():
    geom = GEOMS["c1"]
    G = tnlm.Geometry(geom)
    G.set_stage_timing(True)
    y = cuda(synth.uniform(G.proj_shape, 160))
    f = torch.zeros(G.vol_shape, device="cuda")
    tnlm.tnlm_reconstruct(G, y, f, tnlm.Params(tau=1e-3, n_outer=3, n_inner=2))
    ms, n = G.stage_timing()
    assert n == [6, 6, 3] and all(m > 0 for m in ms)


def test_invalid_arguments_raise():
    G = tnlm.Geometry(GEOMS["c1"])
    f = torch.zeros(G.vol_shape, device="cuda")
    y = torch.zeros(G.proj_shape, device="cuda")
    with pytest.raises(tnlm.TnlmError):
        tnlm.tnlm_reconstruct(G, y, f, tnlm.Params(tau=1e-3, M=7))
    with pytest.raises(tnlm.TnlmError):
        tnlm.tnlm_reconstruct(G, y, f, tnlm.Params(tau=1e-3, n_inner=0))
    with pytest.raises(ValueError):
        tnlm.tnlm_project(G, f.double())


# ---------------------------------------------------------------------------
# full benchmark size (C2: 10 x 256^2 x 64, 36 views x 512 x 384)
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def c2_full():
    pb = synth.recon_problem(synth.C2, device="cuda")
    return pb


def test_full_size_projector_sampled_rays(ora, c2_full):
    pb = c2_full
    G = tnlm.Geometry(pb.geom)
    vol = (pb.truth + torch.from_numpy(synth.normal(G.vol_shape, 170, 0.002)).cuda()).contiguous()
    p = tnlm.tnlm_project(G, vol).cpu().numpy()
    OG = ora.Geometry(pb.geom)
    vh = vol.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(171)
    idx = [(int(rng.integers(G.proj_shape[0])), int(rng.integers(G.proj_shape[2])),
            int(rng.integers(G.proj_shape[1]))) for _ in range(256)]
    got = np.array([p[v, iv, iu] for v, iu, iv in idx])
    ref = np.array([ora.project_ray(OG, vh, v, iu, iv) for v, iu, iv in idx])
    assert rel_l2(got, ref) <= RTOL


def test_full_size_backprojector_adjoint_and_sampled_voxels(ora, c2_full):
    pb = c2_full
    G = tnlm.Geometry(pb.geom)
    y = pb.y
    bt = tnlm.tnlm_backproject(G, y)
    x = (pb.truth + 0.01).contiguous()
    px = tnlm.tnlm_project(G, x)
    lhs = float((px.double() * y.double()).sum())
    rhs = float((x.double() * bt.double()).sum())
    assert abs(lhs - rhs) <= 1e-6 * float(px.double().norm() * y.double().norm())
    OG = ora.Geometry(pb.geom)
    yh = y.cpu().numpy().astype(np.float64)
    bth = bt.cpu().numpy()
    rng = np.random.default_rng(172)
    pts = [(int(rng.integers(10)), int(rng.integers(64)), int(rng.integers(64, 192)), int(rng.integers(64, 192)))
           for _ in range(12)]
    got = np.array([bth[ph, z, yy, xx] for ph, z, yy, xx in pts])
    ref = np.array([ora.backproject_voxel(OG, yh, ph, xx, yy, z) for ph, z, yy, xx in pts])
    assert rel_l2(got, ref) <= RTOL


def test_full_size_sweep_sampled_voxels(ora, c2_full):
    pb = c2_full
    a = (pb.truth + torch.from_numpy(synth.normal(pb.truth.shape, 173, 0.002)).cuda()).contiguous()
    cfg = synth.C2
    out = tnlm.tnlm_gauss_jacobi(a, a, a, cfg.d, cfg.M, cfg.h, cfg.mu, 1).cpu().numpy()
    ah = a.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(174)
    pts = [(int(rng.integers(10)), int(rng.integers(64)), int(rng.integers(256)), int(rng.integers(256)))
           for _ in range(300)]
    got = np.array([out[ph, z, yy, xx] for ph, z, yy, xx in pts])
    ref = np.array([ora.gj_voxel(ah, ah, ah, ph, xx, yy, z, cfg.d, cfg.M, cfg.h, cfg.mu, 1) for ph, z, yy, xx in pts])
    assert rel_l2(got, ref) <= RTOL


def test_sweep_far_beyond_rescale_threshold(ora):
    """Uniform data with h = 0.02 puts c2 D near 10^4: the running references of the online
    normalisation move by far more than the rescale threshold, and no warp skips the rescale
    test.  A volume large enough for interior and boundary tiles of every launch shape; sampled
    voxels (corners, faces and the middle) against the oracle."""
    shape = (3, 24, 40, 72)
    a = synth.uniform(shape, 900)
    v = synth.uniform(shape, 901)
    g = synth.uniform(shape, 902)
    d, M, h, mu = 1, 3, 0.02, 0.8
    out = tnlm.tnlm_gauss_jacobi(cuda(a), cuda(v), cuda(g), d, M, h, mu, 0).cpu().numpy()
    assert np.isfinite(out).all()
    rng = np.random.default_rng(903)
    pts = [(int(rng.integers(3)), int(rng.integers(24)), int(rng.integers(40)), int(rng.integers(72)))
           for _ in range(150)]
    pts += [(0, 0, 0, 0), (1, 23, 39, 71), (2, 12, 20, 36), (1, 0, 20, 71), (2, 23, 0, 36)]
    got = np.array([out[ph, z, yy, xx] for ph, z, yy, xx in pts])
    ref = np.array([ora.gj_voxel(a, v, g, ph, xx, yy, z, d, M, h, mu, 0) for ph, z, yy, xx in pts])
    assert rel_l2(got, ref) <= RTOL


@pytest.fixture(scope="module")
def c3_full():
    g, _ = synth.enhance_input(synth.C3, device="cuda")
    return g.contiguous()


def _crop(a, lo, hi):
    """a[:, z0:z1, y0:y1, x0:x1] for lo = (z0, y0, x0), hi = (z1, y1, x1), clipped to the volume."""
    _, nz, ny, nx = a.shape
    z0, y0, x0 = max(lo[0], 0), max(lo[1], 0), max(lo[2], 0)
    z1, y1, x1 = min(hi[0], nz), min(hi[1], ny), min(hi[2], nx)
    return a[:, z0:z1, y0:y1, x0:x1], (z0, y0, x0)


def test_full_size_enhance_sampled_voxels_and_crop(ora, c3_full):
    """TNLM-E at the full enhancement size (10 x 512^2 x 128, d = 2, M = 3).
    One sweep: 200 sampled voxels, each evaluated by the oracle on a crop of
    radius M + d around it (exact: every patch read and window candidate of
    the voxel lies in the crop, and where the crop meets the volume edge the
    clamping is the volume's).  Two sweeps: an interior 8^3 block (all 10
    phases) against the oracle's two sweeps on that block plus a halo of
    2 (M + d) = 10 voxels, the dependency radius of two sweeps."""
    cfg = synth.C3
    d, M, h, mu = cfg.d, cfg.M, cfg.h, cfg.mu
    g = c3_full
    f1 = tnlm.tnlm_enhance(g, tnlm.Params(d=d, M=M, h=h, mu=mu, n_outer=1, clip_nonneg=0)).cpu()
    gc = g.cpu()
    _, nz, ny, nx = g.shape
    r = M + d
    rng = np.random.default_rng(175)
    got, ref = [], []
    for _ in range(200):
        ph, z, y, x = (int(rng.integers(10)), int(rng.integers(nz)), int(rng.integers(ny)), int(rng.integers(nx)))
        c, (z0, y0, x0) = _crop(gc, (z - r, y - r, x - r), (z + r + 1, y + r + 1, x + r + 1))
        c = c.numpy().astype(np.float64)
        ref.append(ora.gj_voxel(c, c, c, ph, x - x0, y - y0, z - z0, d, M, h, mu, 0))
        got.append(float(f1[ph, z, y, x]))
    assert rel_l2(np.array(got), np.array(ref)) <= RTOL
    f2 = tnlm.tnlm_enhance(g, tnlm.Params(d=d, M=M, h=h, mu=mu, n_outer=2, clip_nonneg=0)).cpu()
    hw, lo = 2 * r, (60, 250, 250)
    c, _ = _crop(gc, (lo[0] - hw, lo[1] - hw, lo[2] - hw), (lo[0] + 8 + hw, lo[1] + 8 + hw, lo[2] + 8 + hw))
    e2 = ora.enhance(c.numpy(), d, M, h, mu, 2)[:, hw:hw + 8, hw:hw + 8, hw:hw + 8]
    got2 = f2[:, lo[0]:lo[0] + 8, lo[1]:lo[1] + 8, lo[2]:lo[2] + 8].numpy()
    assert rel_l2(got2, e2) <= RTOL


def test_full_size_fused_iteration_equals_composed_calls(c2_full):
    """One tnlm_reconstruct iteration in the benchmark's launch configuration
    (fused residual, scaled transpose, sweep with positivity) equals the same
    iteration composed from tnlm_project / tnlm_backproject /
    tnlm_gauss_jacobi."""
    pb = c2_full
    G = tnlm.Geometry(pb.geom)
    cfg = synth.C2
    f0 = (pb.truth * 0.9).contiguous()
    tau = 2e-6
    f = f0.clone()
    tnlm.tnlm_reconstruct(G, pb.y, f, tnlm.Params(d=cfg.d, M=cfg.M, h=cfg.h, mu=cfg.mu, tau=tau, n_outer=1))
    r = tnlm.tnlm_project(G, f0) - pb.y
    g = tnlm.tnlm_backproject(G, r.contiguous(), f0.clone(), alpha=-tau, beta=1.0)
    f2 = tnlm.tnlm_gauss_jacobi(g, g, g, cfg.d, cfg.M, cfg.h, cfg.mu, 1)
    assert rel_l2(f.cpu().numpy(), f2.cpu().numpy()) <= RTOL


@pytest.mark.parametrize("gj_start,n_gj", [(0, 2), (0, 3), (1, 1), (1, 3)])
def test_reconstruct_multi_sweep_p2(ora, gj_start, n_gj):
    """(P2) with n_gj Eq. 8 iterations (weights of g^(k) frozen) against the oracle."""
    geom = GEOMS["ragged_uneven"]
    OG = ora.Geometry(geom)
    G = tnlm.Geometry(geom)
    y = synth.uniform(G.proj_shape, 180) * 0.5
    f0 = synth.smooth_volume(G.vol_shape, 181)
    tau = 1e-4
    ref = ora.reconstruct(OG, y, f0, tau, 1, 2, 0.02, 0.7, 2, clip=1, gj_start=gj_start, n_gj=n_gj)
    f = cuda(f0)
    tnlm.tnlm_reconstruct(G, cuda(y), f, tnlm.Params(d=1, M=2, h=0.02, mu=0.7, tau=tau, n_outer=2, clip_nonneg=1,
                                                     gj_start=gj_start, n_gj=n_gj))
    assert rel_l2(f.cpu().numpy(), ref) <= RTOL


@pytest.mark.parametrize("name", list(GEOMS))
def test_cgls_matches_oracle(ora, name):
    """(P1) by CGLS with per-phase scalars against the FP64 oracle."""
    geom = GEOMS[name]
    G = tnlm.Geometry(geom)
    OG = ora.Geometry(geom)
    x_true = synth.smooth_volume(G.vol_shape, 190)
    y = ora.project(OG, x_true) + synth.normal(G.proj_shape, 191, 1e-3)
    x0 = synth.smooth_volume(G.vol_shape, 192) * 0.5
    ref, rep_ref = ora.cgls(OG, y, x0, 4, with_report=True)
    x = cuda(x0)
    _, rep = tnlm.tnlm_cgls(G, cuda(y), x, 4, report=True)
    assert rel_l2(x.cpu().numpy(), ref) <= RTOL
    np.testing.assert_allclose(rep, rep_ref, rtol=1e-4)
    assert np.all(np.diff(rep) <= 0)


def test_reconstruct_with_cgls_matches_oracle(ora):
    cfg = synth.C1
    pb = synth.recon_problem(cfg)
    OG = ora.Geometry(pb.geom)
    y = pb.y.numpy()
    ref, rep_ref = ora.reconstruct(OG, y, np.zeros(OG.vol_shape), 0.0, cfg.d, cfg.M, cfg.h, cfg.mu, 2, n_inner=3,
                                   p1_cgls=1, with_report=True)
    G = tnlm.Geometry(pb.geom)
    f = torch.zeros(G.vol_shape, device="cuda")
    _, rep = tnlm.tnlm_reconstruct(G, cuda(y), f, tnlm.Params(d=cfg.d, M=cfg.M, h=cfg.h, mu=cfg.mu, n_outer=2,
                                                              n_inner=3, p1_solver=1), report=True)
    assert rel_l2(f.cpu().numpy(), ref) <= RTOL
    np.testing.assert_allclose(rep, rep_ref, rtol=1e-4)


@pytest.mark.parametrize("name", list(GEOMS))
def test_fdk_matches_oracle(ora, name):
    """FDK (ref. 16) of every phase against the FP64 oracle."""
    geom = GEOMS[name]
    G = tnlm.Geometry(geom)
    OG = ora.Geometry(geom)
    objs = [[((1.0, -0.5, 0.3), (6.0, 5.0, 3.0), 0.02), ((-2.0, 1.0, 0.0), (2.0, 2.0, 2.0), 0.01)]
            for _ in range(G.np)]
    p = synth.analytic_projections(geom, objs).numpy() + synth.normal(G.proj_shape, 200, 1e-3)
    ref = ora.fdk(OG, p)
    out = tnlm.tnlm_fdk(G, cuda(p)).cpu().numpy()
    assert rel_l2(out, ref) <= RTOL


BF16_U = 2.0 ** -9  # unit roundoff of bfloat16 (8-bit significand, round to nearest)


@pytest.mark.parametrize("shape,d,M", [((3, 9, 13, 19), 1, 3), ((3, 7, 10, 11), 2, 3), ((2, 8, 12, 20), 2, 1)])
def test_bf16_sweep_is_rounded_fp32_sweep(ora, shape, d, M):
    """BF16 storage / FP32 arithmetic: the sweep on BF16 images equals the
    FP32 sweep on the same (BF16-valued) images rounded to BF16, bit for bit;
    against the FP64 oracle its error is the output rounding (<= 2^-9)."""
    a, v, g, h = _sweep_inputs(shape, 210, "smooth")
    A, V, Gi = (torch.from_numpy(t).cuda().to(torch.bfloat16) for t in (a, v, g))
    out_bf = tnlm.tnlm_gauss_jacobi_bf16(A, V, Gi, d, M, h, 0.8, 1)
    out_f = tnlm.tnlm_gauss_jacobi(A.float().contiguous(), V.float().contiguous(), Gi.float().contiguous(), d, M, h,
                                   0.8, 1)
    assert torch.equal(out_bf, out_f.to(torch.bfloat16))
    ref = ora.gj_sweep(A.float().cpu().numpy(), V.float().cpu().numpy(), Gi.float().cpu().numpy(), d, M, h, 0.8, 1)
    assert rel_l2(out_bf.float().cpu().numpy(), ref) <= BF16_U


def test_bf16_enhance_error_vs_fp64(ora):
    """TNLM-E with BF16 storage over 5 sweeps against the FP64 oracle on the
    same BF16-valued input: each sweep rounds its output (relative <= u) and
    the Jacobi map contracts by 2/(2+mu), so the error stays below u/(1-2/3)."""
    cfg = synth.EnhanceConfig("t", 4, (24, 20, 12), 1.0, 0.002, 0.003, 36, 2, 3, 0.04, 1.0, 5, 220)
    g, _ = synth.enhance_input(cfg)
    G = g.cuda().to(torch.bfloat16)
    p = tnlm.Params(d=2, M=3, h=0.04, mu=1.0, n_outer=5, clip_nonneg=0)
    f = tnlm.tnlm_enhance_bf16(G, p)
    ref = ora.enhance(G.float().cpu().numpy(), 2, 3, 0.04, 1.0, 5)
    err = rel_l2(f.float().cpu().numpy(), ref)
    f32 = tnlm.tnlm_enhance(G.float().contiguous(), p).cpu().numpy()
    err32 = rel_l2(f32, ref)
    print(f"TNLM-E 5 sweeps vs FP64: BF16 storage rel-L2 {err:.3e}, FP32 {err32:.3e}")
    assert err <= 3 * BF16_U
    assert err32 <= RTOL


def _energy_inputs(shape, proj_shape, seed):
    """Independent inputs (an extra case): f and y independent of the weight
    source, so the residual P f - y and the TNLM terms are O(1)."""
    a = synth.smooth_volume(shape, seed)
    f = synth.uniform(shape, seed + 1, 0.0, 0.04)
    y = synth.uniform(proj_shape, seed + 2, 0.0, 0.3)
    return a, f, y


def _phantom_energy_inputs(ora, geom, seed, sigma=5e-4):
    """Phantom-like inputs, the regime of a gradient user near convergence:
    the weight source a is phantom structure, f = a + N(0, sigma^2), so f is
    close to its own weighted means; y = measurements of a with Poisson noise
    at the workloads' photon count I0 = 1e5 (for the C1 geometry its phantom
    and noisy analytic projections; otherwise the oracle's P a made noisy)."""
    if geom is GEOMS["c1"]:
        pb = synth.recon_problem(synth.C1)
        a, y = pb.truth.numpy(), pb.y.numpy()
    else:
        OG = ora.Geometry(geom)
        a = synth.smooth_volume(OG.vol_shape, seed)
        y = synth.poisson_log(torch.from_numpy(ora.project(OG, a)), 1e5, seed + 2).numpy().astype(np.float32)
    f = (a + synth.normal(a.shape, seed + 1, sigma)).astype(np.float32)
    return a, f, y


# An FP32 exact-path projector places each plane crossing of a ray to a few
# units of roundoff times its distance from the isocentre (where the ray
# parameter is anchored): about 1e-6 of the ray's length on these volumes.
# The fidelity half of the gradient, mu P^T (P f - y), is the difference of
# the terms mu P^T P f and mu P^T y, each formed to that accuracy; where the
# residual is far smaller than P f (phantom-like f measured by its own noisy
# projections) the difference is accurate to ~1e-6 of the terms' scale rather
# than of itself.  That is the bound asserted there, besides the 1e-5
# tolerance, which the TNLM half and the well-conditioned cases meet alone.
FIDELITY_EPS = 1e-6


def _fidelity_terms_scale(ora, OG, f, y, mu):
    """||mu P^T P f|| + ||mu P^T y|| from the FP64 oracle."""
    pf = ora.project(OG, f)
    return mu * (np.linalg.norm(ora.backproject(OG, pf)) + np.linalg.norm(ora.backproject(OG, y)))


def _assert_gradient(got, ref, scale, label):
    """rel-L2 <= 1e-5, or an absolute error within FIDELITY_EPS of the
    fidelity terms' scale (the FP32 bound of a small difference of large terms)."""
    err = float(np.linalg.norm(np.asarray(got, np.float64) - ref))
    nref = float(np.linalg.norm(ref))
    print(f"{label}: gradient rel-L2 {err / nref:.2e}; error / fidelity terms' scale {err / scale:.2e} "
          f"(terms' scale / |grad| = {scale / nref:.0f})")
    assert err <= max(RTOL * nref, FIDELITY_EPS * scale)


def _inputs(ora, kind, geom, G, seed):
    if kind == "phantom":
        return _phantom_energy_inputs(ora, geom, seed)
    return _energy_inputs(G.vol_shape, G.proj_shape, seed)


@pytest.mark.parametrize("kind", ["phantom", "independent"])
@pytest.mark.parametrize("name", ["ragged_uneven", "c1"])
def test_energy_grad_matches_oracle(ora, name, kind):
    """E(f) of Eq. 1 (J of Eq. 2, frozen Eq. 9 weights from a) and its
    gradient against the FP64 oracle's scatter-form gradient, on phantom-like
    inputs (f = a + small noise) and on independent ones."""
    geom = GEOMS[name]
    G = tnlm.Geometry(geom)
    OG = ora.Geometry(geom)
    a, f, y = _inputs(ora, kind, geom, G, 230)
    p = tnlm.Params(d=1, M=2, h=0.02, mu=0.7)
    E_ref, g_ref = ora.energy_grad(OG, y, f, a, 1, 2, 0.02, 0.7)
    E, g = tnlm.tnlm_energy_grad(G, cuda(y), cuda(f), cuda(a), p)
    assert E == pytest.approx(E_ref, rel=1e-5)
    if kind == "independent":
        assert rel_l2(g.cpu().numpy(), g_ref) <= RTOL
    else:
        _assert_gradient(g.cpu().numpy(), g_ref, _fidelity_terms_scale(ora, OG, f, y, 0.7), f"{name}/{kind}")
    # the TNLM half alone (fidelity weight negligible) holds the FP32 tolerance on every input
    _, gt_ref = ora.energy_grad(OG, y, f, a, 1, 2, 0.02, 1e-12)
    _, gt = tnlm.tnlm_energy_grad(G, cuda(y), cuda(f), cuda(a), tnlm.Params(d=1, M=2, h=0.02, mu=1e-12))
    assert rel_l2(gt.cpu().numpy(), gt_ref) <= RTOL


@pytest.mark.parametrize("kind", ["phantom", "independent"])
def test_energy_grad_two_phases(ora, kind):
    geom = synth.make_geometry(nx=14, ny=12, nz=9, dx=1.0, nu=30, nv=14, du=1.2, sad=200, sdd=300, n_phases=2,
                               views_per_phase=[5, 6], angle_offset=0.1)
    G = tnlm.Geometry(geom)
    OG = ora.Geometry(geom)
    a, f, y = _inputs(ora, kind, geom, G, 233)
    E_ref, g_ref = ora.energy_grad(OG, y, f, a, 2, 1, 0.03, 1.3)
    E, g = tnlm.tnlm_energy_grad(G, cuda(y), cuda(f), cuda(a), tnlm.Params(d=2, M=1, h=0.03, mu=1.3))
    assert E == pytest.approx(E_ref, rel=1e-5)
    if kind == "independent":
        assert rel_l2(g.cpu().numpy(), g_ref) <= RTOL
    else:
        _assert_gradient(g.cpu().numpy(), g_ref, _fidelity_terms_scale(ora, OG, f, y, 1.3), f"two phases/{kind}")
    _, gt_ref = ora.energy_grad(OG, y, f, a, 2, 1, 0.03, 1e-12)
    _, gt = tnlm.tnlm_energy_grad(G, cuda(y), cuda(f), cuda(a), tnlm.Params(d=2, M=1, h=0.03, mu=1e-12))
    assert rel_l2(gt.cpu().numpy(), gt_ref) <= RTOL


def test_energy_grad_tnlm_part_near_fixed_point(ora):
    """The TNLM half alone where cancellation would show: the fidelity weight
    is made negligible (mu = 1e-12), a is smooth structure of small contrast
    and f = a + 1e-5 noise, so f is within ~1e-3 of its weighted means and the
    gradient is ~1e-3 of f.  A form such as f (1 + sum w) - sum w f_j would
    lose ~u |f| / |grad| ~ 4e-5 here; each pair contributing its own
    difference keeps the FP32 tolerance."""
    geom = GEOMS["c1"]
    G = tnlm.Geometry(geom)
    OG = ora.Geometry(geom)
    a = synth.smooth_volume(G.vol_shape, 236, amp=5e-4)
    f = (a + synth.normal(a.shape, 237, 1e-5)).astype(np.float32)
    y = np.zeros(G.proj_shape, np.float32)
    E_ref, g_ref = ora.energy_grad(OG, y, f, a, 1, 2, 0.02, 1e-12)
    E, g = tnlm.tnlm_energy_grad(G, cuda(y), cuda(f), cuda(a), tnlm.Params(d=1, M=2, h=0.02, mu=1e-12))
    scale = float(np.linalg.norm(g_ref) / np.linalg.norm(f))
    err = rel_l2(g.cpu().numpy(), g_ref)
    print(f"|grad| / |f| = {scale:.1e}, rel-L2 {err:.2e}")
    assert scale < 3e-3
    assert err <= RTOL
    assert E == pytest.approx(E_ref, rel=1e-5)


@pytest.mark.parametrize("d, M", [(1, 2), (2, 1), (1, 3)])
def test_energy_grad_bf16_equals_fp32_on_widened_inputs(d, M):
    """BF16 storage of y, f and a: every value is widened before use and the
    gradient is FP32, so the call equals the FP32 call on the widened inputs
    bit for bit (energy and gradient)."""
    geom = GEOMS["ragged_uneven"]
    G = tnlm.Geometry(geom)
    a, f, y = _energy_inputs(G.vol_shape, G.proj_shape, 240)
    a16, f16, y16 = cuda(a).bfloat16(), cuda(f).bfloat16(), cuda(y).bfloat16()
    p = tnlm.Params(d=d, M=M, h=0.03, mu=0.7)
    E16, g16 = tnlm.tnlm_energy_grad_bf16(G, y16, f16, a16, p)
    E32, g32 = tnlm.tnlm_energy_grad(G, y16.float(), f16.float(), a16.float(), p)
    torch.cuda.synchronize()
    assert E16 == E32
    assert torch.equal(g16, g32)


@pytest.mark.parametrize("kind", ["phantom", "independent"])
def test_energy_autograd_and_directional_derivatives(ora, kind):
    """TNLMEnergy in autograd: f.grad is the kernels' gradient, and along 64
    random directions it matches FP64 central differences of the oracle's
    energy."""
    geom = GEOMS["c1"]
    G = tnlm.Geometry(geom)
    OG = ora.Geometry(geom)
    a, f0, y = _inputs(ora, kind, geom, G, 235)
    p = tnlm.Params(d=1, M=2, h=0.02, mu=0.7)
    f = cuda(f0).requires_grad_(True)
    E = tnlm.TNLMEnergy.apply(f, G, cuda(y), cuda(a), p)
    (2.0 * E).backward()
    _, g = tnlm.tnlm_energy_grad(G, cuda(y), cuda(f0), cuda(a), p)
    assert torch.allclose(f.grad, 2.0 * g)
    gh = g.double().cpu().numpy()
    _, g_ref = ora.energy_grad(OG, y, f0, a, 1, 2, 0.02, 0.7)
    _assert_gradient(gh, g_ref, _fidelity_terms_scale(ora, OG, f0, y, 0.7), f"autograd/{kind}")
    rng = np.random.default_rng(237)
    eps = 1e-4
    for _ in range(64):
        v = rng.standard_normal(G.vol_shape)
        fd = (ora.energy_grad(OG, y, f0 + eps * v, a, 1, 2, 0.02, 0.7)[0] -
              ora.energy_grad(OG, y, f0 - eps * v, a, 1, 2, 0.02, 0.7)[0]) / (2 * eps)
        assert float((gh * v).sum()) == pytest.approx(fd, rel=1e-4)


@pytest.fixture(scope="module")
def c4_full():
    pb = synth.recon_problem(synth.C4, device="cuda")
    return synth.ReconProblem(pb.cfg, pb.geom, pb.truth.cpu(), pb.y.cpu())


def test_full_size_energy_grad_sampled_voxels(ora, c4_full):
    """The differentiable-energy workload at its own size (10 x 128^3 at 2 mm,
    40 views x 256 x 192, patch 3^3, window 5^3), phantom-like f = a + noise
    with a the phantom and y its noisy projections.  On 40 sampled voxels
    (faces and corners included) the gradient is compared with the oracle's:
    the fidelity half mu (P^T (P f - y))(x) from the oracle's full FP64
    residual and its plain-definition transpose at x, the TNLM half from the
    oracle on a crop of radius 2M + d around x (exact: pass 0 reads within
    M + d of x; the transposed term weighs candidates y within M of x by
    normalisers that read within M + d of y; where the crop meets the volume
    edge the clamping and window validity are the volume's).  The TNLM half
    alone holds 1e-5; the whole gradient holds 1e-5 or FIDELITY_EPS of its
    fidelity terms' scale, mu (|P^T P f| + |P^T y|) at the sampled voxels."""
    cfg = synth.C4
    pb = c4_full
    d, M, h, mu = cfg.d, cfg.M, cfg.h, cfg.mu
    a = pb.truth.numpy()
    f = (a + synth.normal(a.shape, 300, 5e-4)).astype(np.float32)
    y = pb.y.numpy()
    G = tnlm.Geometry(pb.geom)
    _, g = tnlm.tnlm_energy_grad(G, cuda(y), cuda(f), cuda(a), tnlm.Params(d=d, M=M, h=h, mu=mu))
    g = g.cpu().numpy()
    _, gt_gpu = tnlm.tnlm_energy_grad(G, cuda(y), cuda(f), cuda(a), tnlm.Params(d=d, M=M, h=h, mu=1e-12))
    gt_gpu = gt_gpu.cpu().numpy()
    G.close()
    OG = ora.Geometry(pb.geom)
    pf = ora.project(OG, f)
    r = pf - y
    np_, nz, ny, nx = a.shape
    rng = np.random.default_rng(301)
    pts = [(int(rng.integers(np_)), int(rng.integers(nz)), int(rng.integers(ny)), int(rng.integers(nx)))
           for _ in range(32)]
    pts += [(0, 0, 0, 0), (3, nz - 1, ny - 1, nx - 1), (5, 0, ny // 2, nx - 1), (9, nz - 1, 0, nx // 2),
            (1, 1, 64, 2), (7, 126, 3, 64), (2, 64, 64, 64), (8, 2, 125, 1)]
    R = 2 * M + d
    got, ref, got_t, ref_t, t_pf, t_y = [], [], [], [], [], []
    for ph, z, yy, x in pts:
        c_a, (z0, y0, x0) = _crop(a, (z - R, yy - R, x - R), (z + R + 1, yy + R + 1, x + R + 1))
        c_f, _ = _crop(f, (z - R, yy - R, x - R), (z + R + 1, yy + R + 1, x + R + 1))
        cg = synth.make_geometry(nx=c_a.shape[3], ny=c_a.shape[2], nz=c_a.shape[1], dx=2.0, nu=1, nv=1, du=1.0,
                                 n_phases=np_, views_per_phase=1)
        OC = ora.Geometry(cg)
        _, gt = ora.energy_grad(OC, np.zeros(OC.proj_shape), c_f, c_a, d, M, h, 0.0)
        fid = mu * ora.backproject_voxel(OG, r, ph, x, yy, z)
        ref.append(fid + gt[ph, z - z0, yy - y0, x - x0])
        got.append(float(g[ph, z, yy, x]))
        ref_t.append(gt[ph, z - z0, yy - y0, x - x0])
        got_t.append(float(gt_gpu[ph, z, yy, x]))
        t_pf.append(mu * ora.backproject_voxel(OG, pf, ph, x, yy, z))
        t_y.append(mu * ora.backproject_voxel(OG, y, ph, x, yy, z))
    err_t = rel_l2(np.array(got_t), np.array(ref_t))
    print(f"config-4 sampled: TNLM half alone rel-L2 {err_t:.2e}; "
          f"|TNLM half| / |gradient| {np.linalg.norm(ref_t) / np.linalg.norm(ref):.2e}")
    assert err_t <= RTOL
    _assert_gradient(np.array(got), np.array(ref), float(np.linalg.norm(t_pf) + np.linalg.norm(t_y)),
                     "config-4 sampled")


def _weight_grad_inputs(shape, seed):
    """a: smooth + noise (distances D/2h^2 of order 1 for the h used), f
    independent of a so that q varies across the window."""
    a = synth.smooth_volume(shape, seed) + synth.normal(shape, seed + 1, 0.01)
    f = synth.uniform(shape, seed + 2, 0.0, 0.04)
    return a, f


@pytest.mark.parametrize("shape, d, M, h", [((3, 20, 18, 11), 1, 2, 0.05),  # ragged tiles (8 x 8 x 4)
                                             ((2, 9, 10, 7), 2, 1, 0.1),     # N_p = 2, d = 2
                                             ((4, 33, 17, 9), 1, 3, 0.06),   # M = 3
                                             ((2, 6, 5, 1), 1, 1, 0.05)])    # a single slice
def test_energy_grad_weights_matches_oracle(ora, shape, d, M, h):
    """Gradient of 1/2 sum J through the Eq. 9 weights (w.r.t. the weight
    source a) against the FP64 oracle's scatter form."""
    a, f = _weight_grad_inputs(shape, 260)
    ref = ora.energy_grad_a(f, a, d, M, h)
    got = tnlm.tnlm_energy_grad_weights(cuda(f), cuda(a), d, M, h)
    assert rel_l2(got.cpu().numpy(), ref) <= RTOL


def test_energy_autograd_weights_differentiated(ora):
    """TNLMEnergy with the weights computed from f itself: f.grad is the
    frozen-weight gradient plus the gradient through the weights, equal to
    the oracle's (and, in the oracle, to central differences of E(f))."""
    geom = GEOMS["c1"]
    G = tnlm.Geometry(geom)
    OG = ora.Geometry(geom)
    f0 = synth.smooth_volume(G.vol_shape, 262) * 0.02 + synth.uniform(G.vol_shape, 263, 0.0, 0.02)
    y = synth.uniform(G.proj_shape, 264, 0.0, 0.3)
    d, M, h, mu = 1, 2, 0.03, 0.7
    p = tnlm.Params(d=d, M=M, h=h, mu=mu)
    f = cuda(f0).requires_grad_(True)
    E = tnlm.TNLMEnergy.apply(f, G, cuda(y), f, p)
    E.backward()
    E_ref, gf = ora.energy_grad(OG, y, f0, f0, d, M, h, mu)
    ref = gf + ora.energy_grad_a(f0, f0, d, M, h)
    assert float(E.detach()) == pytest.approx(E_ref, rel=1e-5)
    assert rel_l2(f.grad.cpu().numpy(), ref) <= RTOL
    # frozen: a detached gives the f-gradient alone
    f2 = cuda(f0).requires_grad_(True)
    tnlm.TNLMEnergy.apply(f2, G, cuda(y), f2.detach(), p).backward()
    assert rel_l2(f2.grad.cpu().numpy(), gf) <= RTOL


def test_reconstruct_batch_graph_equals_single_calls():
    """Uneven problems in one captured graph replayed n_outer times give the
    same images, bit for bit, as separate tnlm_reconstruct calls."""
    geoms = [GEOMS["ragged_uneven"], synth.C1.geometry(),
             synth.make_geometry(nx=20, ny=18, nz=10, dx=1.5, nu=40, nv=24, du=1.2, sad=300, sdd=450, n_phases=5,
                                 views_per_phase=[6, 7, 5, 8, 6], angle_offset=0.07)]
    params = [tnlm.Params(d=1, M=2, h=0.02, mu=0.8, tau=1e-4, n_outer=3),
              tnlm.Params(d=1, M=2, h=0.02, mu=1.0, n_outer=3, n_inner=2, p1_solver=1),
              tnlm.Params(d=2, M=1, h=0.03, mu=1.2, tau=5e-5, n_outer=3, n_gj=2)]
    Gs = [tnlm.Geometry(g) for g in geoms]
    ys = [cuda(synth.uniform(G.proj_shape, 240 + k) * 0.3) for k, G in enumerate(Gs)]
    f0 = [synth.smooth_volume(G.vol_shape, 250 + k) for k, G in enumerate(Gs)]
    single = []
    for G, y, f, p in zip(Gs, ys, f0, params):
        x = cuda(f)
        tnlm.tnlm_reconstruct(G, y, x, p)
        single.append(x)
    Gb = [tnlm.Geometry(g) for g in geoms]
    fb = [cuda(f) for f in f0]
    tnlm.tnlm_reconstruct_batch(Gb, ys, fb, params)
    torch.cuda.synchronize()
    for a, b in zip(single, fb):
        assert torch.equal(a, b)
    # the reusable plan: replays of 2 and then 1 iteration continue from f
    fp = [cuda(f) for f in f0]
    plan = tnlm.BatchPlan(Gb, ys, fp, params)
    plan.run(2)
    plan.run(1)
    plan.close()
    torch.cuda.synchronize()
    for a, b in zip(single, fp):
        assert torch.equal(a, b)


def _batch_oracle_problems(ora, n_outer):
    """Uneven TNLM-R problems with the batched workload's structure at reduced
    sizes (the oracle runs each in seconds): uneven views within a problem,
    different volumes, detectors and phase counts, a gradient-step problem, a
    CGLS one (n_inner = 2) and a multi-sweep one (d = 2, M = 1, n_gj = 2 from
    f^(k-1)); tau = 1/L from the oracle's power iteration."""
    thorax = synth.ReconConfig("reduced batch problem", 6, (32, 32, 12), 16.0, [5, 6, 7, 5, 6, 8], (48, 36), 8.3,
                               5e4, 1, 3, 0.02, 1.0, n_outer, "thorax", 2100)
    pb = synth.recon_problem(thorax)
    geoms = [GEOMS["ragged_uneven"], synth.C1.geometry(),
             synth.make_geometry(nx=20, ny=18, nz=10, dx=1.5, nu=40, nv=24, du=1.2, sad=300, sdd=450, n_phases=5,
                                 views_per_phase=[6, 7, 5, 8, 6], angle_offset=0.07),
             pb.geom]
    ys = [synth.uniform(ora.Geometry(geoms[0]).proj_shape, 241) * 0.3, synth.recon_problem(synth.C1).y.numpy(),
          synth.uniform(ora.Geometry(geoms[2]).proj_shape, 242) * 0.3, pb.y.numpy()]
    params = [dict(d=1, M=2, h=0.02, mu=0.8), dict(d=1, M=2, h=0.02, mu=1.0, n_inner=2, p1_solver=1),
              dict(d=2, M=1, h=0.03, mu=1.2, n_gj=2, gj_start=1), dict(d=1, M=3, h=0.02, mu=1.0)]
    out = []
    for k, (geom, y, pp) in enumerate(zip(geoms, ys, params)):
        OG = ora.Geometry(geom)
        tau = float(np.float32(1.0 / ora.power_norm(OG, synth.uniform(OG.vol_shape, 90 + k), 30)))
        out.append((geom, OG, np.asarray(y, np.float32), tnlm.Params(tau=tau, n_outer=n_outer, **pp)))
    return out


def _oracle_recon(ora, OG, y, p):
    return ora.reconstruct(OG, y, np.zeros(OG.vol_shape), p.tau, p.d, p.M, p.h, p.mu, p.n_outer, n_inner=p.n_inner,
                           clip=p.clip_nonneg, gj_start=p.gj_start, n_gj=p.n_gj, p1_cgls=p.p1_solver)


def test_reconstruct_batch_matches_oracle(ora):
    """Every problem of an uneven batch, run as one captured graph
    (tnlm_reconstruct_batch) and as a reusable plan replayed in two parts,
    against the FP64 oracle's TNLM-R after 20 iterations: relative L2 <= 1e-5
    per problem."""
    n_outer = 20
    probs = _batch_oracle_problems(ora, n_outer)
    refs = [_oracle_recon(ora, OG, y, p) for _, OG, y, p in probs]
    Gs = [tnlm.Geometry(geom) for geom, _, _, _ in probs]
    ys = [cuda(y) for _, _, y, _ in probs]
    params = [p for _, _, _, p in probs]
    fb = [torch.zeros(G.vol_shape, device="cuda") for G in Gs]
    tnlm.tnlm_reconstruct_batch(Gs, ys, fb, params)
    fp = [torch.zeros(G.vol_shape, device="cuda") for G in Gs]
    plan = tnlm.BatchPlan(Gs, ys, fp, params)
    plan.run(12)
    plan.run(n_outer - 12)
    plan.close()
    torch.cuda.synchronize()
    for k, (a, b, ref) in enumerate(zip(fb, fp, refs)):
        err = rel_l2(a.cpu().numpy(), ref)
        print(f"batch problem {k}: rel-L2 vs FP64 {err:.2e}")
        assert err <= RTOL
        assert torch.equal(a, b)


def test_batch_plan_bf16_error_vs_fp64(ora):
    """The same uneven batch (the gradient-step and multi-sweep problems; BF16
    storage runs (P1) as gradient steps) in BF16 storage, 20 iterations,
    against the FP64 oracle on the same BF16-representable measurements: per
    problem within 2 n_outer u (u = 2^-9, two roundings per iteration), and the
    measured maximum is printed."""
    n_outer = 20
    probs = [pr for pr in _batch_oracle_problems(ora, n_outer) if pr[3].p1_solver == 0]
    ys = [_bf16_round(y) for _, _, y, _ in probs]
    refs = [_oracle_recon(ora, OG, y, p) for (_, OG, _, p), y in zip(probs, ys)]
    Gs = [tnlm.Geometry(geom) for geom, _, _, _ in probs]
    f16 = [torch.zeros(G.vol_shape, device="cuda", dtype=torch.bfloat16) for G in Gs]
    plan = tnlm.BatchPlan(Gs, [cuda(y).bfloat16() for y in ys], f16, [p for _, _, _, p in probs])
    plan.run(n_outer)
    plan.close()
    torch.cuda.synchronize()
    errs = [rel_l2(f.float().cpu().numpy(), ref) for f, ref in zip(f16, refs)]
    print(f"BF16 batch, {n_outer} iterations: rel-L2 vs FP64 per problem {[f'{e:.2e}' for e in errs]}, "
          f"max {max(errs):.2e}")
    assert max(errs) <= 2 * n_outer * BF16_U


def _bf16_round(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).bfloat16().float().numpy()


@pytest.mark.parametrize("cfg, n_outer", [(synth.C1, synth.C1.n_outer), (C2_TINY, 10)])
def test_reconstruct_bf16_error_vs_fp64(ora, cfg, n_outer):
    """TNLM-R with BF16 storage against the FP64 oracle on the same
    (BF16-representable) measurements.  Each iteration rounds g and f to BF16
    once (unit roundoff u = 2^-9 each) and the gradient step with tau <= 1/L
    and the averaging sweep do not amplify earlier errors much, so the error
    stays within 2 n_outer u; the measured value is far below that bound."""
    pb = synth.recon_problem(cfg)
    OG = ora.Geometry(pb.geom)
    L = ora.power_norm(OG, synth.uniform(OG.vol_shape, 7), 30)
    tau = float(np.float32(1.0 / L))
    y = _bf16_round(pb.y.numpy())
    f_ref, rep_ref = ora.reconstruct(OG, y, np.zeros(OG.vol_shape), tau, cfg.d, cfg.M, cfg.h, cfg.mu, n_outer,
                                     with_report=True)
    G = tnlm.Geometry(pb.geom)
    p = tnlm.Params(d=cfg.d, M=cfg.M, h=cfg.h, mu=cfg.mu, tau=tau, n_outer=n_outer)
    f16 = torch.zeros(G.vol_shape, device="cuda", dtype=torch.bfloat16)
    _, rep = tnlm.tnlm_reconstruct_bf16(G, cuda(y).bfloat16(), f16, p, report=True)
    f32 = torch.zeros(G.vol_shape, device="cuda")
    tnlm.tnlm_reconstruct(G, cuda(y), f32, p)
    err16 = rel_l2(f16.float().cpu().numpy(), f_ref)
    err32 = rel_l2(f32.cpu().numpy(), f_ref)
    print(f"BF16 storage rel-L2 vs FP64 after {n_outer} iterations: {err16:.3e} (FP32: {err32:.1e})")
    assert err32 <= RTOL
    assert err16 <= 2 * n_outer * BF16_U
    np.testing.assert_allclose(rep, rep_ref, rtol=4 * n_outer * BF16_U)
    assert torch.all(f16.float() >= 0)


def test_batch_plan_bf16_equals_single_calls():
    """BF16 problems in one captured plan equal separate BF16 calls bit for bit."""
    geoms = [GEOMS["ragged_uneven"], synth.C1.geometry()]
    params = [tnlm.Params(d=1, M=2, h=0.02, mu=0.8, tau=1e-4, n_outer=2),
              tnlm.Params(d=2, M=1, h=0.03, mu=1.1, tau=5e-5, n_outer=2, n_gj=2, gj_start=1)]
    Gs = [tnlm.Geometry(g) for g in geoms]
    ys = [cuda(synth.uniform(G.proj_shape, 270 + k) * 0.3).bfloat16() for k, G in enumerate(Gs)]
    f0 = [cuda(synth.smooth_volume(G.vol_shape, 280 + k)).bfloat16() for k, G in enumerate(Gs)]
    single = []
    for G, y, f, p in zip(Gs, ys, f0, params):
        x = f.clone()
        tnlm.tnlm_reconstruct_bf16(G, y, x, p)
        single.append(x)
    Gb = [tnlm.Geometry(g) for g in geoms]
    fb = [f.clone() for f in f0]
    plan = tnlm.BatchPlan(Gb, ys, fb, params)
    plan.run(2)
    plan.close()
    torch.cuda.synchronize()
    for a, b in zip(single, fb):
        assert torch.equal(a, b)


def test_out_of_memory_paths_and_recovery(ora):
    """Device allocations made to fail on the host (the library's test hook,
    no GPU fault): tnlm_reconstruct and tnlm_enhance return 'out of device
    memory' before launching anything and the same handle then works and
    gives the normal result; a failed transpose prefix workspace falls back
    to the exact per-cell transpose, still equal to the oracle."""
    lib = tnlm._load()
    pb = synth.recon_problem(synth.C1)
    p = tnlm.Params(d=1, M=2, h=0.02, mu=1.0, tau=1e-3, n_outer=2)
    G = tnlm.Geometry(pb.geom)
    f = torch.zeros(G.vol_shape, device="cuda")
    tnlm.tnlm_project(G, f)  # builds the handle's projector tables first
    assert lib.tnlm_test_fail_allocations(1) == 0
    with pytest.raises(tnlm.TnlmError) as e:
        tnlm.tnlm_reconstruct(G, cuda(pb.y.numpy()), f, p)
    assert e.value.status == 3 and "failed" in str(e.value)
    assert torch.count_nonzero(f) == 0
    tnlm.tnlm_reconstruct(G, cuda(pb.y.numpy()), f, p)
    G2 = tnlm.Geometry(pb.geom)
    f2 = torch.zeros(G2.vol_shape, device="cuda")
    tnlm.tnlm_reconstruct(G2, cuda(pb.y.numpy()), f2, p)
    torch.cuda.synchronize()
    assert torch.equal(f, f2)
    # projector tables that cannot be allocated: the slab walker runs, equal to the oracle
    G4 = tnlm.Geometry(GEOMS["ragged_uneven"])
    x = synth.uniform(G4.vol_shape, 78)
    assert lib.tnlm_test_fail_allocations(1) == 0
    px = tnlm.tnlm_project(G4, cuda(x)).cpu().numpy()
    assert lib.tnlm_test_fail_allocations(0) == 0
    assert tnlm.tnlm_get_launch_shapes(G4)["projector_rows"] == 4
    assert rel_l2(px, ora.project(ora.Geometry(GEOMS["ragged_uneven"]), x)) <= RTOL
    G4.close()
    g = cuda(synth.smooth_volume((3, 8, 12, 16), 5))
    pe = tnlm.Params(d=1, M=1, h=0.02, mu=1.0, n_outer=3, clip_nonneg=0)
    assert lib.tnlm_test_fail_allocations(1) == 0
    with pytest.raises(tnlm.TnlmError) as e:
        tnlm.tnlm_enhance(g, pe)
    assert e.value.status == 3
    ref = ora.enhance(g.cpu().numpy(), 1, 1, 0.02, 1.0, 3)
    assert rel_l2(tnlm.tnlm_enhance(g, pe).cpu().numpy(), ref) <= RTOL
    # transpose without its prefix workspace: the exact per-cell form
    geom = GEOMS["ragged_uneven"]
    G3 = tnlm.Geometry(geom)
    proj = synth.uniform(G3.proj_shape, 77)
    assert lib.tnlm_test_fail_allocations(1) == 0
    bt = tnlm.tnlm_backproject(G3, cuda(proj)).cpu().numpy()
    assert lib.tnlm_test_fail_allocations(0) == 0
    assert rel_l2(bt, ora.backproject(ora.Geometry(geom), proj)) <= RTOL
    for h in (G, G2, G3):
        h.close()


def test_reconstruct_resumes_from_its_iterate():
    """TNLM-R keeps no state between iterations besides f (the weights are
    recomputed from g^(k) every iteration), so resuming from a saved iterate
    is a second call: 3 + 2 iterations equal 5 bit for bit."""
    pb = synth.recon_problem(synth.C1)
    y = cuda(pb.y.numpy())
    G = tnlm.Geometry(pb.geom)
    f5 = torch.zeros(G.vol_shape, device="cuda")
    tnlm.tnlm_reconstruct(G, y, f5, tnlm.Params(d=1, M=2, h=0.02, mu=1.0, tau=1e-3, n_outer=5))
    f = torch.zeros(G.vol_shape, device="cuda")
    tnlm.tnlm_reconstruct(G, y, f, tnlm.Params(d=1, M=2, h=0.02, mu=1.0, tau=1e-3, n_outer=3))
    saved = f.cpu()
    f = saved.cuda()
    tnlm.tnlm_reconstruct(G, y, f, tnlm.Params(d=1, M=2, h=0.02, mu=1.0, tau=1e-3, n_outer=2))
    torch.cuda.synchronize()
    assert torch.equal(f, f5)
    G.close()


def test_grouped_persistent_sweep_equals_per_problem_plan(ora):
    """Uneven problems sharing (d, M) = (1, 3): the plan whose sweeps run as one
    persistent launch (CTAs taking (problem, tile) items from a device
    counter) gives the per-problem plan's images bit for bit, and the oracle's
    TNLM-R to 1e-5."""
    cfgs = [synth.ReconConfig("grouped batch problem", nph, vol, 512.0 / vol[0], views, det, 399.4 / det[0], 5e4,
                              1, 3, 0.02, 1.0, 3, "thorax", 2200 + k)
            for k, (nph, vol, views, det) in enumerate([(3, (32, 32, 12), [5, 6, 4], (48, 36)),
                                                        (4, (40, 40, 16), [4, 5, 6, 5], (64, 48)),
                                                        (2, (24, 24, 9), [6, 5], (40, 30))])]
    probs = [synth.recon_problem(c) for c in cfgs]
    params = []
    for k, pb in enumerate(probs):
        OG = ora.Geometry(pb.geom)
        tau = float(np.float32(1.0 / ora.power_norm(OG, synth.uniform(OG.vol_shape, 800 + k), 30)))
        params.append(tnlm.Params(d=1, M=3, h=0.02, mu=1.0, tau=tau, n_outer=3))
    Gs = [tnlm.Geometry(pb.geom) for pb in probs]
    ys = [cuda(pb.y.numpy()) for pb in probs]
    f_plain = [torch.zeros(G.vol_shape, device="cuda") for G in Gs]
    f_group = [torch.zeros(G.vol_shape, device="cuda") for G in Gs]
    p1 = tnlm.BatchPlan(Gs, ys, f_plain, params)
    p1.run(3)
    p1.close()
    p2 = tnlm.BatchPlan(Gs, ys, f_group, params, grouped=True)
    p2.run(2)
    p2.run(1)
    p2.close()
    torch.cuda.synchronize()
    for a, b in zip(f_plain, f_group):
        assert torch.equal(a, b)
    pb, p = probs[1], params[1]
    ref = ora.reconstruct(ora.Geometry(pb.geom), pb.y.numpy(), np.zeros(Gs[1].vol_shape), p.tau, 1, 3, 0.02, 1.0, 3)
    assert rel_l2(f_group[1].cpu().numpy(), ref) <= RTOL


@pytest.mark.parametrize("name, shape", [("ragged_uneven", 104), ("ragged_uneven", 4), ("c1", 104)])
def test_reconstruct_host_equals_device_call(name, shape):
    """tnlm_reconstruct_host (phase-by-phase copies from pinned host memory, the first projection
    started per phase as its copy lands) against tnlm_reconstruct on the same inputs: f and the
    residual report bit for bit, with the table and the slab walker; CGLS (no per-phase start) and
    n_outer = 0 (f copied there and back)."""
    G = tnlm.Geometry(GEOMS[name])
    tnlm.tnlm_set_launch_shapes(G, shape, 8, 4)
    y = synth.uniform(G.proj_shape, 880) * 0.3
    f0 = synth.smooth_volume(G.vol_shape, 881)
    L = tnlm.tnlm_operator_norm(G, cuda(synth.uniform(G.vol_shape, 882)), 20)
    cases = [tnlm.Params(d=1, M=2, h=0.02, mu=0.7, tau=1.0 / L, n_outer=2, n_inner=2, clip_nonneg=1),
             tnlm.Params(d=1, M=2, h=0.02, mu=0.7, n_outer=1, n_inner=2, p1_solver=1),
             tnlm.Params(d=1, M=2, h=0.02, mu=0.7, tau=1.0 / L, n_outer=0)]
    for p in cases:
        f_dev_ref = cuda(f0)
        _, rep_ref = tnlm.tnlm_reconstruct(G, cuda(y), f_dev_ref, p, report=True)
        y_host = torch.from_numpy(np.ascontiguousarray(y, np.float32)).pin_memory()
        f_host = torch.from_numpy(np.ascontiguousarray(f0, np.float32)).pin_memory()
        y_dev = torch.full(G.proj_shape, float("nan"), device="cuda")
        f_dev = torch.full(G.vol_shape, float("nan"), device="cuda")
        *_, rep = tnlm.reconstruct_host(G, y_host, f_host, p, y_dev, f_dev, report=True)
        torch.cuda.synchronize()
        assert torch.equal(f_host, f_dev_ref.cpu())
        assert torch.equal(f_dev, f_dev_ref)
        assert np.array_equal(rep, rep_ref)
    G.close()
