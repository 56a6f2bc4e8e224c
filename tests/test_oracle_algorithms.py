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


def test_reconstruct_multi_sweep_p2(ora):
    """n_gj Eq. 8 iterations per (P2) with the weights of g^(k) frozen, the
    positivity correction after the last one."""
    geom, truth, y = _small_problem(50)
    G = ora.Geometry(geom)
    tau, d, M, h, mu = 0.01, 1, 1, 0.05, 0.8
    f0 = truth.astype(np.float64)
    for gj_start in (0, 1):
        f = ora.reconstruct(G, y, f0, tau, d, M, h, mu, n_outer=1, n_gj=3, clip=1, gj_start=gj_start)
        g = f0 - tau * ora.backproject(G, ora.project(G, f0) - y)
        w = ora.weights(g, d, M, h)
        fl = f0.copy() if gj_start else g.copy()
        for l in range(3):
            fl = ora.gj_apply(w, M, fl, g, mu, clip=1 if l == 2 else 0)
        np.testing.assert_allclose(f, fl, rtol=1e-12, atol=1e-15)


def test_cgls_reaches_least_squares_and_is_phase_separable(ora):
    """CGLS (ref. 37) on an overdetermined tiny problem reaches the dense
    least-squares solution; residuals never grow; running it on all phases at
    once equals running it on each phase alone (Sec. 2.3: (P1) is uncoupled)."""
    geom = synth.make_geometry(nx=4, ny=4, nz=3, dx=1.0, nu=10, nv=6, du=1.2, sad=30, sdd=45, n_phases=2,
                               views_per_phase=[5, 4], angle_offset=0.1)
    G = ora.Geometry(geom)
    x_true = synth.smooth_volume(G.vol_shape, 60).astype(np.float64)
    y = ora.project(G, x_true) + synth.normal(G.proj_shape, 61, 1e-3)
    x, rep = ora.cgls(G, y, np.zeros(G.vol_shape), 200, with_report=True)
    assert np.all(np.diff(rep) <= 1e-12 * rep[0])
    # dense least squares per phase
    nvox = 48
    for ph, (v0, v1) in enumerate(((0, 5), (5, 9))):
        sub = dict(geom)
        sub["nviews"] = np.array([v1 - v0], np.int32)
        sub["angles"] = np.asarray(geom["angles"][v0:v1])
        Gs = ora.Geometry(sub)
        cols = []
        for v in range(nvox):
            e = np.zeros((1, 3, 4, 4))
            e.reshape(-1)[v] = 1.0
            cols.append(ora.project(Gs, e).ravel())
        P = np.stack(cols, 1)
        x_ls = np.linalg.lstsq(P, y[v0:v1].ravel(), rcond=None)[0]
        np.testing.assert_allclose(x[ph].ravel(), x_ls, rtol=1e-6, atol=1e-8)
        # a few iterations on the phase alone equal the joint run's iterates
        xa = ora.cgls(Gs, y[v0:v1], np.zeros((1, 3, 4, 4)), 5)
        xj = ora.cgls(G, y, np.zeros(G.vol_shape), 5)
        np.testing.assert_allclose(xj[ph], xa[0], rtol=1e-11, atol=1e-14)


def test_reconstruct_with_cgls_p1(ora):
    geom, truth, y = _small_problem(62)
    G = ora.Geometry(geom)
    d, M, h, mu = 1, 1, 0.05, 0.8
    f0 = truth.astype(np.float64)
    f, rep = ora.reconstruct(G, y, f0, 0.0, d, M, h, mu, n_outer=1, n_inner=3, p1_cgls=1, with_report=True)
    g, crep = ora.cgls(G, y, f0, 3, with_report=True)
    np.testing.assert_allclose(rep[0], crep[:3], rtol=1e-12)
    np.testing.assert_allclose(f, ora.gj_sweep(g, g, g, d, M, h, mu, 1), rtol=1e-12, atol=1e-15)


def test_fdk_reconstructs_known_balls(ora):
    """FDK (ref. 16) of analytic projections: phase 0 holds a centred ball,
    phase 1 an off-centre one; each phase's FDK from its own 180 views
    recovers its own ball's attenuation in the core and ~0 outside."""
    import torch
    n = 40
    geom = synth.make_geometry(nx=n, ny=n, nz=16, dx=1.0, nu=96, nv=40, du=1.0, sad=300, sdd=450, n_phases=2,
                               views_per_phase=180)
    balls = [((0.0, 0.0, 0.0), 10.0, 0.02), ((5.0, -4.0, 2.0), 6.0, 0.03)]
    objs = [[(c, (r, r, r), m)] for c, r, m in balls]
    p = synth.analytic_projections(geom, objs).numpy()
    f = ora.fdk(ora.Geometry(geom), p)
    xs = np.arange(n) - 0.5 * (n - 1)
    zs = np.arange(16) - 7.5
    for ph, (c, r, m) in enumerate(balls):
        d2 = (xs[None, None, :] - c[0]) ** 2 + (xs[None, :, None] - c[1]) ** 2 + (zs[:, None, None] - c[2]) ** 2
        core = d2 < (0.6 * r) ** 2
        out = d2 > (r + 4.0) ** 2
        assert abs(f[ph][core].mean() - m) < 0.005 * m, (ph, f[ph][core].mean())
        assert abs(f[ph][out].mean()) < 0.01 * m


def test_energy_gradient_finite_differences(ora):
    """The oracle's total energy (Eq. 1, J of Eq. 2, frozen Eq. 9 weights)
    equals its parts, and its gradient matches FP64 central differences along
    64 random directions."""
    geom, truth, y = _small_problem(70)
    G = ora.Geometry(geom)
    f = truth.astype(np.float64) + synth.normal(G.vol_shape, 71, 0.002)
    a = truth.astype(np.float64)
    d, M, h, mu = 1, 1, 0.02, 0.7
    E, grad = ora.energy_grad(G, y, f, a, d, M, h, mu)
    w = ora.weights(a, d, M, h)
    assert E == pytest.approx(0.5 * mu * ora.fidelity(G, f, y) + 0.5 * ora.tnlm_energy(w, M, f), rel=1e-12)
    rng = np.random.default_rng(72)
    eps = 1e-4
    for _ in range(64):
        v = rng.standard_normal(G.vol_shape)
        fd = (ora.energy_grad(G, y, f + eps * v, a, d, M, h, mu)[0] -
              ora.energy_grad(G, y, f - eps * v, a, d, M, h, mu)[0]) / (2 * eps)
        assert fd == pytest.approx(float((grad * v).sum()), rel=1e-7, abs=1e-12)


def _tnlm_half(ora, f, a, d, M, h):
    return 0.5 * ora.tnlm_energy(ora.weights(a, d, M, h), M, f)


@pytest.mark.parametrize("shape, d, M, h", [((3, 5, 6, 7), 1, 1, 0.05), ((2, 4, 5, 6), 1, 2, 0.08),
                                             ((4, 4, 4, 5), 2, 1, 0.12)])
def test_energy_gradient_through_weights_finite_differences(ora, shape, d, M, h):
    """The weights differentiated: the oracle's gradient of 1/2 sum J (Eq. 2,
    weights of Eq. 9 from a) with respect to a matches FP64 central
    differences of that energy along 48 random directions; boundary clamping,
    N_p = 2 (both directions to the same phase) and d = 2 included."""
    f = synth.smooth_volume(shape, 80) + synth.normal(shape, 81, 0.01)
    a = synth.smooth_volume(shape, 82) + synth.normal(shape, 83, 0.01)
    g = ora.energy_grad_a(f, a, d, M, h)
    assert np.abs(g).max() > 0
    rng = np.random.default_rng(84)
    eps = 1e-6  # truncation error ~eps^2 (checked: 2.5e-4, 2.5e-6, 2.5e-8 relative at 1e-3, 1e-4, 1e-5)
    for _ in range(48):
        v = rng.standard_normal(shape)
        fd = (_tnlm_half(ora, f, a + eps * v, d, M, h) - _tnlm_half(ora, f, a - eps * v, d, M, h)) / (2 * eps)
        assert fd == pytest.approx(float((g * v).sum()), rel=1e-6, abs=1e-10)


def test_self_weighted_energy_gradient(ora):
    """With the weights computed from f itself, the total gradient of Eq. 1 is
    the frozen-weight gradient plus the gradient through the weights (chain
    rule); checked against central differences of E(f) = mu/2 ||Pf - y||^2 +
    1/2 sum J[f; w(f)] along 32 random directions."""
    geom, truth, y = _small_problem(85)
    G = ora.Geometry(geom)
    f = truth.astype(np.float64) + synth.normal(G.vol_shape, 86, 0.003)
    d, M, h, mu = 1, 1, 0.03, 0.6

    def energy(x):
        return 0.5 * mu * ora.fidelity(G, x, y) + _tnlm_half(ora, x, x, d, M, h)

    E, gf = ora.energy_grad(G, y, f, f, d, M, h, mu)
    assert E == pytest.approx(energy(f), rel=1e-12)
    grad = gf + ora.energy_grad_a(f, f, d, M, h)
    rng = np.random.default_rng(87)
    eps = 1e-6
    for _ in range(32):
        v = rng.standard_normal(G.vol_shape)
        fd = (energy(f + eps * v) - energy(f - eps * v)) / (2 * eps)
        assert fd == pytest.approx(float((grad * v).sum()), rel=1e-6, abs=1e-10)
