"""Pins of the oracle's projector P and its transpose against facts fixed
independently of the oracle: closed-form chords, a dense matrix built by a
separate slab computation, the adjoint identity, the half-open cell rule, an
SVD, and analytic ellipsoid line integrals (Sec. 2.5 uses Siddon's exact
radiological path for P)."""
import math

import numpy as np
import pytest
import torch

from paper_1201_2450_gb300 import synth


def _rays(geom):
    """(source, pixel) endpoints of every ray, written out from the geometry
    convention (phase-major views, u fastest)."""
    out = []
    for th in geom["angles"]:
        c, s = math.cos(th), math.sin(th)
        for iv in range(geom["nv"]):
            for iu in range(geom["nu"]):
                u = (iu - 0.5 * (geom["nu"] - 1)) * geom["du"] + geom["u_off"]
                v = (iv - 0.5 * (geom["nv"] - 1)) * geom["dv"] + geom["v_off"]
                src = np.array([geom["sad"] * c, geom["sad"] * s, 0.0])
                pix = np.array([(geom["sad"] - geom["sdd"]) * c - u * s, (geom["sad"] - geom["sdd"]) * s + u * c, v])
                out.append((src, pix))
    return out


def _slab_chords(src, pix, lo, hi):
    """Vectorised slab-method chord of segments (src->pix) [R,3] through boxes
    [lo, hi) [V,3] -> [R, V] (mm)."""
    d = (pix - src)[:, None, :]
    s = src[:, None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        a0 = (lo[None] - s) / d
        a1 = (hi[None] - s) / d
    lo_a = np.where(d == 0, np.where((s >= lo[None]) & (s < hi[None]), -np.inf, np.inf), np.minimum(a0, a1))
    hi_a = np.where(d == 0, np.where((s >= lo[None]) & (s < hi[None]), np.inf, -np.inf), np.maximum(a0, a1))
    amin = np.maximum(lo_a.max(axis=2), 0.0)
    amax = np.minimum(hi_a.min(axis=2), 1.0)
    return np.clip(amax - amin, 0.0, None) * np.linalg.norm(pix - src, axis=1)[:, None]


def _voxel_boxes(geom):
    nx, ny, nz = geom["nx"], geom["ny"], geom["nz"]
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    lo = np.stack([geom["cx"] + (ix.ravel() - 0.5 * nx) * geom["dx"],
                   geom["cy"] + (iy.ravel() - 0.5 * ny) * geom["dy"],
                   geom["cz"] + (iz.ravel() - 0.5 * nz) * geom["dz"]], axis=1)
    return lo, lo + np.array([geom["dx"], geom["dy"], geom["dz"]])


def _dense_P(ora, geom):
    """Dense P of the oracle, one column per unit voxel image."""
    G = ora.Geometry(geom)
    nvox = geom["nx"] * geom["ny"] * geom["nz"]
    cols = []
    for ph in range(G.np):
        for v in range(nvox):
            e = np.zeros(G.vol_shape)
            e.reshape(G.np, -1)[ph, v] = 1.0
            cols.append(ora.project(G, e).ravel())
    return np.stack(cols, axis=1), G


TINY = synth.make_geometry(nx=4, ny=3, nz=2, dx=1.0, dy=1.3, dz=0.9, cx=0.2, cy=-0.1, cz=0.05, nu=7, nv=5,
                           du=0.9, dv=1.1, u_off=0.13, v_off=-0.07, sad=20.0, sdd=32.0, n_phases=2,
                           views_per_phase=3, angle_offset=0.1)


def test_dense_matrix_equals_slab_chords(ora):
    """Every element of P is the exact chord of that ray through that cell."""
    P, G = _dense_P(ora, TINY)
    rays = _rays(TINY)
    src = np.array([r[0] for r in rays])
    pix = np.array([r[1] for r in rays])
    lo, hi = _voxel_boxes(TINY)
    chords = _slab_chords(src, pix, lo, hi)  # [rays, nvox]
    nvox = lo.shape[0]
    npix = TINY["nu"] * TINY["nv"]
    expect = np.zeros_like(P)
    v0 = 0
    for ph, nview in enumerate(TINY["nviews"]):
        rows = slice(v0 * npix, (v0 + nview) * npix)
        expect[rows, ph * nvox:(ph + 1) * nvox] = chords[rows]
        v0 += nview
    assert np.count_nonzero(expect) > 50
    np.testing.assert_allclose(P, expect, rtol=1e-12, atol=1e-12)
    # the oracle's own slab chord agrees with the same closed form
    for r in (0, 17, 40):
        for v in (0, 5, 23):
            assert ora.chord(lo[v], hi[v], src[r], pix[r]) == pytest.approx(chords[r, v], rel=1e-12, abs=1e-13)


def test_constant_volume_is_box_chord(ora):
    geom = synth.make_geometry(nx=9, ny=7, nz=5, dx=1.0, nu=16, nv=12, du=1.5, sad=40, sdd=60, n_phases=2,
                               views_per_phase=4, angle_offset=0.05)
    G = ora.Geometry(geom)
    c = 0.37
    p = ora.project(G, np.full(G.vol_shape, c))
    rays = _rays(geom)
    src = np.array([r[0] for r in rays])
    pix = np.array([r[1] for r in rays])
    lo = np.array([[-4.5, -3.5, -2.5]])
    chords = _slab_chords(src, pix, lo, -lo)[:, 0]
    np.testing.assert_allclose(p.ravel(), c * chords, rtol=1e-12, atol=1e-12)
    assert (chords > 0).sum() > 100


def test_axis_aligned_ray_closed_form(ora):
    """The central ray at angle 0 runs along -x at y = z = 0 (odd ny, nz: the
    row's voxel centres), so it integrates dx * sum_x f over that row."""
    geom = synth.make_geometry(nx=6, ny=5, nz=3, dx=1.25, nu=5, nv=3, du=1.0, sad=30, sdd=45, n_phases=2,
                               views_per_phase=1, angles=[0.0, 0.5])
    G = ora.Geometry(geom)
    f = synth.uniform(G.vol_shape, 3).astype(np.float64)
    p = ora.project(G, f)
    assert p[0, 1, 2] == pytest.approx(1.25 * f[0, 1, 2, :].sum(), rel=1e-13)


def test_ray_in_face_plane_half_open(ora):
    """Even ny: y = 0 is the face between rows ny/2-1 and ny/2.  A ray lying in
    that plane belongs to the cell whose lower face it lies in (row ny/2)."""
    geom = synth.make_geometry(nx=6, ny=4, nz=3, dx=1.0, nu=5, nv=3, du=1.0, sad=30, sdd=45, n_phases=2,
                               views_per_phase=1, angles=[0.0, 0.5])
    G = ora.Geometry(geom)
    f = synth.uniform(G.vol_shape, 4).astype(np.float64)
    p = ora.project(G, f)
    assert p[0, 1, 2] == pytest.approx(f[0, 1, 2, :].sum(), rel=1e-13)
    assert p[0, 1, 2] != pytest.approx(f[0, 1, 1, :].sum(), rel=1e-6)


def test_adjoint_identity_fp64(ora):
    geom = synth.make_geometry(nx=12, ny=10, nz=6, dx=1.0, nu=20, nv=12, du=1.3, sad=50, sdd=75, n_phases=3,
                               views_per_phase=[4, 5, 3])
    G = ora.Geometry(geom)
    x = synth.uniform(G.vol_shape, 5).astype(np.float64)
    y = synth.uniform(G.proj_shape, 6).astype(np.float64)
    lhs = float((ora.project(G, x) * y).sum())
    rhs = float((x * ora.backproject(G, y)).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_backproject_scatter_equals_plain_definition(ora):
    """The ray-driven scatter equals sum_rays r * |ray ∩ cell| at every voxel."""
    geom = synth.make_geometry(nx=5, ny=4, nz=3, dx=1.0, nu=9, nv=6, du=1.2, sad=30, sdd=45, n_phases=2,
                               views_per_phase=3, angle_offset=0.2)
    G = ora.Geometry(geom)
    y = synth.uniform(G.proj_shape, 7).astype(np.float64)
    bt = ora.backproject(G, y)
    for ph in range(2):
        for iz in range(3):
            for iy in range(4):
                for ix in range(5):
                    assert ora.backproject_voxel(G, y, ph, ix, iy, iz) == pytest.approx(bt[ph, iz, iy, ix],
                                                                                          rel=1e-11, abs=1e-12)


def test_power_norm_matches_svd(ora):
    P, G = _dense_P(ora, TINY)
    smax2 = np.linalg.svd(P, compute_uv=False)[0] ** 2
    x0 = synth.uniform(G.vol_shape, 8).astype(np.float64)
    L = ora.power_norm(G, x0, 400)
    # block-diagonal P: phases with nearly equal top singular values make the
    # Rayleigh quotient converge slowly, but it is always a lower bound
    assert L == pytest.approx(smax2, rel=1e-4)
    assert L <= smax2 * (1 + 1e-12)


def test_projector_approximates_analytic_phantom(ora):
    """P of a point-sampled ellipsoid phantom converges to its analytic line
    integrals as the grid is refined (only discretisation error remains)."""
    objs = synth._small_objects(2)
    errs = []
    for n in (24, 96):
        cfg = synth.ReconConfig("t", 2, (n, n, n), 32.0 / n, 3, (40, 30), 2.0, 1e5, 1, 1, 0.02, 1.0, 1, "small", 5)
        geom = cfg.geometry()
        truth = synth.rasterize(geom, objs, dtype=torch.float64).numpy()
        p_ana = synth.analytic_projections(geom, objs).numpy()
        p_vox = ora.project(ora.Geometry(geom), truth)
        errs.append(np.linalg.norm(p_vox - p_ana) / np.linalg.norm(p_ana))
    assert errs[1] < 0.05 and errs[1] < 0.6 * errs[0], errs


def test_ray_in_outer_face_half_open(ora):
    """A ray lying exactly in the volume's lower y face is inside (row 0); one
    lying in the upper y face is outside (projection 0)."""
    for cy, expect_row in ((2.0, 0), (-2.0, None)):
        geom = synth.make_geometry(nx=6, ny=4, nz=3, dx=1.0, cy=cy, nu=5, nv=3, du=1.0, sad=30, sdd=45,
                                   n_phases=2, views_per_phase=1, angles=[0.0, 0.5])
        G = ora.Geometry(geom)
        f = synth.uniform(G.vol_shape, 9).astype(np.float64)
        p = ora.project(G, f)
        if expect_row is None:
            assert p[0, 1, 2] == 0.0
        else:
            assert p[0, 1, 2] == pytest.approx(f[0, 1, expect_row, :].sum(), rel=1e-13)
