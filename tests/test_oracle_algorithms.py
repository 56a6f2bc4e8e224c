"""Pins of the oracle's TNLM-R and TNLM-E loops (Sec. 2.3 algorithm boxes):
each equals its steps composed by hand, (P1) gradient steps with
tau <= 1/||P||^2 never raise the data residual, and TNLM-E keeps constants."""
import numpy as np
import pytest

from paper_1201_2450_gb300 import synth


def _small_problem(seed=40):
    geom = synth.make_geometry(nx=10, ny=9, nz=6, dx=1.0, nu=16, nv=10, du=1.4, sad=40, sdd=60, n_phases=3,
                               views_per_phase=[5, 4, 6])
    nviews = int(np.sum(geom["nviews"]))
    truth = synth.smooth_volume((3, 6, 9, 10), seed)
    y = synth.uniform((nviews, 10, 16), seed + 1) * 0.1
    return geom, truth, y


def test_reconstruct_is_its_steps(ora):
    geom, truth, y = _small_problem()
    G = ora.Geometry(geom)
    L = ora.power_norm(G, synth.uniform(G.vol_shape, 41), 60)
    tau, d, M, h, mu = 1.0 / L, 1, 1, 0.05, 0.8
    f0 = truth.astype(np.float64)
    f, rep = ora.reconstruct(G, y, f0, tau, d, M, h, mu, n_outer=2, n_inner=2, clip=1, with_report=True)
    # by hand: P1 from f^(k-1), weights from g, Eq. 8 with vals = g, clip
    fk = f0.copy()
    for k in range(2):
        g = fk.copy()
        for t in range(2):
            r = ora.project(G, g) - y
            assert rep[k, t] == pytest.approx(float((r * r).sum()), rel=1e-12)
            g = g - tau * ora.backproject(G, r)
        fk = ora.gj_sweep(g, g, g, d, M, h, mu, clip=1)
    np.testing.assert_allclose(f, fk, rtol=1e-12, atol=1e-15)
    assert np.all(f >= 0)


def test_reconstruct_gj_start_previous(ora):
    geom, truth, y = _small_problem(43)
    G = ora.Geometry(geom)
    tau, d, M, h, mu = 0.01, 1, 1, 0.05, 0.8
    f0 = truth.astype(np.float64)
    f = ora.reconstruct(G, y, f0, tau, d, M, h, mu, n_outer=1, n_inner=1, clip=0, gj_start=1)
    g = f0 - tau * ora.backproject(G, ora.project(G, f0) - y)
    np.testing.assert_allclose(f, ora.gj_sweep(g, f0, g, d, M, h, mu), rtol=1e-12, atol=1e-15)


def test_p1_gradient_steps_descend(ora):
    geom, truth, y = _small_problem(44)
    G = ora.Geometry(geom)
    L = ora.power_norm(G, synth.uniform(G.vol_shape, 45), 60)
    _, rep = ora.reconstruct(G, y, np.zeros(G.vol_shape), 1.0 / L, 1, 1, 0.05, 1.0, n_outer=1, n_inner=6,
                             with_report=True)
    assert np.all(np.diff(rep[0]) <= 0), rep


def test_enhance_is_its_sweeps(ora):
    shape = (3, 5, 6, 7)
    g = synth.smooth_volume(shape, 46) + synth.normal(shape, 47, 0.002)
    d, M, h, mu = 1, 1, 0.01, 1.0
    f = ora.enhance(g, d, M, h, mu, 3)
    fk = g.astype(np.float64)
    for _ in range(3):
        fk = ora.gj_sweep(fk, fk, g, d, M, h, mu)
    np.testing.assert_allclose(f, fk, rtol=1e-13)


def test_enhance_constant_and_noise_reduction(ora):
    shape = (4, 6, 6, 6)
    c = np.full(shape, 0.3)
    np.testing.assert_allclose(ora.enhance(c, 1, 1, 0.01, 1.0, 4), c, rtol=1e-14)
    clean = synth.smooth_volume(shape, 48)
    g = clean + synth.normal(shape, 49, 0.002)
    f = ora.enhance(g, 1, 2, 0.01, 1.0, 5)
    assert np.linalg.norm(f - clean) < 0.8 * np.linalg.norm(g - clean)
