"""Seeded synthetic inputs for the TNLM 4D-CBCT path.

This module only *generates inputs*: scan geometry descriptions, phantoms,
their projections and noise.  It holds none of the method's arithmetic (no
voxel projector, no weights, no Gauss-Jacobi update), so both the CUDA
library's tests and the CPU oracle may consume its outputs.

Inputs stand in for the paper's NCAT phantom and clinical scan (Sec. 2.5),
which are not available: they keep the protocol's structure -- phase-
interleaved circular cone-beam views, a thorax-like ellipsoid phantom with a
moving tumour -- and their projections are *analytic* ellipsoid line
integrals (not the voxel model), followed by Poisson noise, so the
reconstruction problem is not an inverse crime.

Geometry convention (shared by the description only): rotation about z,
source at SAD (cos t, sin t, 0), detector centre at (SAD-SDD)(cos t, sin t, 0),
u = (-sin t, cos t, 0), v = (0, 0, 1); pixel (iu, iv) centre at
((iu-(nu-1)/2) du + u_off, (iv-(nv-1)/2) dv + v_off); voxel centres at
((ix-(nx-1)/2) dx + cx, ...).  Projection j of J = Np*V views has angle
2*pi*j/J and belongs to phase j mod Np; views are stored phase-major.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

# --------------------------------------------------------------------------
# scan geometry descriptions
# --------------------------------------------------------------------------


def interleaved_angles(n_phases: int, views_per_phase) -> tuple[np.ndarray, np.ndarray]:
    """Phase-major view angles for a phase-interleaved 360-degree scan.

    ``views_per_phase`` is an int or a per-phase list (uneven bins allowed;
    then the J = sum(V_i) angles are still interleaved round-robin)."""
    if np.isscalar(views_per_phase):
        nviews = np.full(n_phases, int(views_per_phase), np.int32)
    else:
        nviews = np.asarray(views_per_phase, np.int32)
    J = int(nviews.sum())
    # round-robin assignment of equally spaced angles to phases
    owner = []
    left = nviews.copy()
    j = 0
    while len(owner) < J:
        i = j % n_phases
        if left[i] > 0:
            owner.append(i)
            left[i] -= 1
        j += 1
    theta = 2.0 * np.pi * np.arange(J, dtype=np.float64) / J
    owner = np.asarray(owner)
    angles = np.concatenate([theta[owner == i] for i in range(n_phases)])
    return nviews, angles


def make_geometry(*, nx, ny, nz, dx, dy=None, dz=None, cx=0.0, cy=0.0, cz=0.0, nu, nv, du, dv=None,
                  u_off=0.0, v_off=0.0, sad=1000.0, sdd=1500.0, n_phases, views_per_phase,
                  angles=None, angle_offset=0.0) -> dict:
    """Plain-dict geometry description consumed by both the CUDA binding and
    the oracle binding."""
    if angles is None:
        nviews, ang = interleaved_angles(n_phases, views_per_phase)
    else:
        nviews = np.full(n_phases, int(views_per_phase), np.int32) if np.isscalar(views_per_phase) \
            else np.asarray(views_per_phase, np.int32)
        ang = np.asarray(angles, np.float64)
    return dict(nx=int(nx), ny=int(ny), nz=int(nz), dx=float(dx), dy=float(dy if dy is not None else dx),
                dz=float(dz if dz is not None else dx), cx=float(cx), cy=float(cy), cz=float(cz),
                nu=int(nu), nv=int(nv), du=float(du), dv=float(dv if dv is not None else du),
                u_off=float(u_off), v_off=float(v_off), sad=float(sad), sdd=float(sdd),
                nviews=nviews, angles=ang + float(angle_offset))


# --------------------------------------------------------------------------
# workload configurations (the paper's protocol shapes, Sec. 2.5)
# --------------------------------------------------------------------------


@dataclass
class ReconConfig:
    """A TNLM-R workload: geometry + phantom + TNLM parameters."""
    name: str
    n_phases: int
    vol: tuple  # (nx, ny, nz)
    voxel_mm: float
    views_per_phase: object
    det: tuple  # (nu, nv)
    pixel_mm: float
    i0: float
    d: int
    M: int
    h: float
    mu: float
    n_outer: int
    phantom: str  # "small" | "thorax"
    seed: int
    sad: float = 1000.0
    sdd: float = 1500.0
    extra: dict = field(default_factory=dict)

    def geometry(self) -> dict:
        nx, ny, nz = self.vol
        nu, nv = self.det
        return make_geometry(nx=nx, ny=ny, nz=nz, dx=self.voxel_mm, nu=nu, nv=nv, du=self.pixel_mm,
                             sad=self.sad, sdd=self.sdd, n_phases=self.n_phases,
                             views_per_phase=self.views_per_phase)


# 4 phases, 32^3 at 1 mm, 20 views/phase on 64x48 at 1.5 mm, patch 3^3, window 5^3, 5 iterations
C1 = ReconConfig("plain TNLM-R FP32 4x32^3, 20 views x 64x48", 4, (32, 32, 32), 1.0, 20, (64, 48), 1.5,
                 1e5, 1, 2, 0.02, 1.0, 5, "small", 1001)
# 10 phases, 256x256x64 at 2 mm, 36 views/phase on 512x384 at 0.78 mm, patch 3^3, window 7^3, 50 iterations
C2 = ReconConfig("NCAT-shaped TNLM-R FP32 10x256x256x64, 36 views x 512x384", 10, (256, 256, 64), 2.0, 36,
                 (512, 384), 0.78, 5e4, 1, 3, 0.02, 1.0, 50, "thorax", 1002)
# differentiable-energy workload: 10 phases, 128^3 at 2 mm, 40 views/phase on 256x192 at 1.56 mm
C4 = ReconConfig("differentiable energy 10x128^3, 40 views x 256x192", 10, (128, 128, 128), 2.0, 40, (256, 192),
                 1.56, 5e4, 1, 2, 0.02, 1.0, 1, "thorax", 1004)
# reduced C2 with the same structure, for full-length parity runs
C2_SMALL = ReconConfig("NCAT-shaped TNLM-R reduced 10x64x64x16, 9 views x 128x96", 10, (64, 64, 16), 8.0, 9,
                       (128, 96), 3.12, 5e4, 1, 3, 0.02, 1.0, 50, "thorax", 1002)


@dataclass
class EnhanceConfig:
    name: str
    n_phases: int
    vol: tuple
    voxel_mm: float
    noise_sigma: float
    streak_amp: float
    n_streaks: int
    d: int
    M: int
    h: float
    mu: float
    n_sweeps: int
    seed: int


# 10 x 512^2 x 128, patch 5^3, window 7^3, 30 sweeps
C3 = EnhanceConfig("TNLM-E FP32 10x512x512x128", 10, (512, 512, 128), 1.0, 0.002, 0.003, 36, 2, 3, 0.04, 1.0, 30,
                   1003)
C3_SMALL = EnhanceConfig("TNLM-E reduced 10x64x64x16", 10, (64, 64, 16), 8.0, 0.002, 0.003, 36, 2, 3, 0.04, 1.0,
                         30, 1003)


# --------------------------------------------------------------------------
# ellipsoid phantoms
# --------------------------------------------------------------------------


def _small_objects(n_phases: int, scale=(1.0, 1.0, 1.0)):
    """C1-style phantom (mm): body, two lungs, a tumour moving +-3 mm in z.
    Each object is (centre, semi-axes, delta-mu) and the image is the sum of
    delta-mu over the objects containing a point (nested layers)."""
    sx, sy, sz = scale
    out = []
    for i in range(n_phases):
        dz = 3.0 * math.sin(2.0 * math.pi * i / n_phases)
        objs = [((0.0, 0.0, 0.0), (14.0, 11.0, 14.0), 0.02),
                ((-6.5, 0.0, 0.0), (5.0, 7.0, 10.0), 0.004 - 0.02),
                ((6.5, 0.0, 0.0), (5.0, 7.0, 10.0), 0.004 - 0.02),
                ((6.5, 0.0, dz), (4.0, 4.0, 4.0), 0.02 - 0.004)]
        out.append([((c[0] * sx, c[1] * sy, c[2] * sz), (a[0] * sx, a[1] * sy, a[2] * sz), m) for c, a, m in objs])
    return out


def _thorax_objects(n_phases: int, scale: float = 1.0):
    """C2-style thorax (mm): body with +-2 mm AP chest-wall motion, lungs,
    heart, spine (mu 0.04), tumour moving +-8 mm in z."""
    out = []
    for i in range(n_phases):
        ph = math.sin(2.0 * math.pi * i / n_phases)
        objs = [((0.0, 0.0, 0.0), (125.0, 90.0 + 2.0 * ph, 60.0), 0.02),
                ((-60.0, 0.0, 0.0), (35.0, 50.0, 45.0), 0.004 - 0.02),
                ((60.0, 0.0, 0.0), (35.0, 50.0, 45.0), 0.004 - 0.02),
                ((0.0, -40.0, -10.0), (22.0, 25.0, 25.0), 0.022 - 0.02),
                ((0.0, 65.0, 0.0), (12.0, 12.0, 60.0), 0.04 - 0.02),
                ((55.0, 10.0, 8.0 * ph), (10.0, 10.0, 10.0), 0.02 - 0.004)]
        out.append([((c[0] * scale, c[1] * scale, c[2] * scale), tuple(x * scale for x in a), m) for c, a, m in objs])
    return out


def _objects(cfg: ReconConfig):
    if cfg.phantom == "small":
        # C1 geometry is 32 mm wide; scale the phantom to other grids
        ext = np.array(cfg.vol) * cfg.voxel_mm / 32.0
        return _small_objects(cfg.n_phases, tuple(ext))
    ext = cfg.vol[0] * cfg.voxel_mm / 512.0
    return _thorax_objects(cfg.n_phases, ext)


def rasterize(geom: dict, objects_per_phase, device="cpu", dtype=torch.float32) -> torch.Tensor:
    """Point-sample the layered ellipsoid phantom at voxel centres."""
    nx, ny, nz = geom["nx"], geom["ny"], geom["nz"]
    dev = torch.device(device)
    xs = (torch.arange(nx, device=dev, dtype=torch.float64) - 0.5 * (nx - 1)) * geom["dx"] + geom["cx"]
    ys = (torch.arange(ny, device=dev, dtype=torch.float64) - 0.5 * (ny - 1)) * geom["dy"] + geom["cy"]
    zs = (torch.arange(nz, device=dev, dtype=torch.float64) - 0.5 * (nz - 1)) * geom["dz"] + geom["cz"]
    vols = []
    for objs in objects_per_phase:
        v = torch.zeros((nz, ny, nx), dtype=torch.float64, device=dev)
        for (c, a, m) in objs:
            q = (((xs - c[0]) / a[0]) ** 2)[None, None, :] + (((ys - c[1]) / a[1]) ** 2)[None, :, None] + \
                (((zs - c[2]) / a[2]) ** 2)[:, None, None]
            v += m * (q <= 1.0)
        vols.append(v)
    return torch.stack(vols).to(dtype)


def analytic_projections(geom: dict, objects_per_phase, device="cpu") -> torch.Tensor:
    """Exact line integrals of the layered ellipsoid phantom along every
    source->pixel segment (FP64), shape [sum views][nv][nu]."""
    dev = torch.device(device)
    nu, nv = geom["nu"], geom["nv"]
    u = (torch.arange(nu, device=dev, dtype=torch.float64) - 0.5 * (nu - 1)) * geom["du"] + geom["u_off"]
    v = (torch.arange(nv, device=dev, dtype=torch.float64) - 0.5 * (nv - 1)) * geom["dv"] + geom["v_off"]
    V, U = torch.meshgrid(v, u, indexing="ij")
    sad, sdd = geom["sad"], geom["sdd"]
    out = torch.empty((len(geom["angles"]), nv, nu), dtype=torch.float64, device=dev)
    vg = 0
    for ph, nview in enumerate(geom["nviews"]):
        for _ in range(int(nview)):
            th = float(geom["angles"][vg])
            c, s = math.cos(th), math.sin(th)
            src = (sad * c, sad * s, 0.0)
            px = (sad - sdd) * c - U * s
            py = (sad - sdd) * s + U * c
            pz = V
            d = (px - src[0], py - src[1], pz - src[2])
            dl = torch.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
            acc = torch.zeros_like(U)
            for (cc, a, m) in objects_per_phase[ph]:
                o = [(src[k] - cc[k]) / a[k] for k in range(3)]
                e = [d[k] / a[k] for k in range(3)]
                A = e[0] ** 2 + e[1] ** 2 + e[2] ** 2
                B = 2.0 * (o[0] * e[0] + o[1] * e[1] + o[2] * e[2])
                Cc = o[0] ** 2 + o[1] ** 2 + o[2] ** 2 - 1.0
                disc = B * B - 4.0 * A * Cc
                sq = torch.sqrt(torch.clamp(disc, min=0.0))
                t1 = (-B - sq) / (2.0 * A)
                t2 = (-B + sq) / (2.0 * A)
                L = torch.clamp(torch.minimum(t2, torch.ones_like(t2)) - torch.clamp(t1, min=0.0), min=0.0)
                acc += m * torch.where(disc > 0, L * dl, torch.zeros_like(L))
            out[vg] = acc
            vg += 1
    return out


def poisson_log(p: torch.Tensor, i0: float, seed: int) -> torch.Tensor:
    """y = ln(I0 / max(N, 1)) with N ~ Poisson(I0 exp(-p)), seeded."""
    gen = torch.Generator(device=p.device)
    gen.manual_seed(seed)
    lam = i0 * torch.exp(-p)
    n = torch.poisson(lam, generator=gen)
    return torch.log(i0 / torch.clamp(n, min=1.0))


@dataclass
class ReconProblem:
    cfg: ReconConfig
    geom: dict
    truth: torch.Tensor  # [Np][nz][ny][nx] float32
    y: torch.Tensor  # [sum views][nv][nu] float32


def recon_problem(cfg: ReconConfig, device="cpu", noise=True) -> ReconProblem:
    """Phantom, analytic projections and Poisson noise for a TNLM-R config."""
    geom = cfg.geometry()
    objs = _objects(cfg)
    truth = rasterize(geom, objs, device=device)
    p = analytic_projections(geom, objs, device=device)
    y = poisson_log(p, cfg.i0, cfg.seed) if noise else p
    return ReconProblem(cfg, geom, truth, y.to(torch.float32))


def enhance_input(cfg: EnhanceConfig, device="cpu") -> tuple[torch.Tensor, torch.Tensor]:
    """(noisy streaked input g, clean phantom) for a TNLM-E config: C1-style
    phantom scaled to the grid + N(0, sigma^2) + per-phase radial streaks
    amp*cos(n_streaks*(atan2(y,x) - phi_i)), phi_i ~ U[0, 2 pi / n_streaks)."""
    nx, ny, nz = cfg.vol
    geom = make_geometry(nx=nx, ny=ny, nz=nz, dx=cfg.voxel_mm, nu=2, nv=2, du=1.0, n_phases=cfg.n_phases,
                         views_per_phase=1)
    ext = np.array(cfg.vol) * cfg.voxel_mm / 32.0
    clean = rasterize(geom, _small_objects(cfg.n_phases, tuple(ext)), device=device)
    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(cfg.seed)
    phi = torch.rand(cfg.n_phases, generator=gen, device=dev, dtype=torch.float64) * (2 * math.pi / cfg.n_streaks)
    xs = (torch.arange(nx, device=dev, dtype=torch.float64) - 0.5 * (nx - 1)) * cfg.voxel_mm
    ys = (torch.arange(ny, device=dev, dtype=torch.float64) - 0.5 * (ny - 1)) * cfg.voxel_mm
    ang = torch.atan2(ys[:, None], xs[None, :])
    g = clean.clone()
    for i in range(cfg.n_phases):
        streak = cfg.streak_amp * torch.cos(cfg.n_streaks * (ang - phi[i]))
        noise = torch.randn((nz, ny, nx), generator=gen, device=dev, dtype=torch.float32) * cfg.noise_sigma
        g[i] += streak.to(torch.float32)[None, :, :] + noise
    return g, clean


# --------------------------------------------------------------------------
# plain random inputs for operator tests
# --------------------------------------------------------------------------


def uniform(shape, seed: int, lo=0.0, hi=1.0) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, size=shape).astype(np.float32)


def normal(shape, seed: int, sigma=1.0) -> np.ndarray:
    return (np.random.default_rng(seed).standard_normal(size=shape) * sigma).astype(np.float32)


def smooth_volume(shape, seed: int, n_blobs=6, base=0.02, amp=0.01) -> np.ndarray:
    """Sum of random Gaussian blobs (+ base) on an (Np, nz, ny, nx) grid --
    smooth structure that shifts a little between phases."""
    rng = np.random.default_rng(seed)
    np_, nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    out = np.full(shape, base, np.float64)
    centres = rng.uniform(0, 1, size=(n_blobs, 3)) * np.array([nx, ny, nz])
    widths = rng.uniform(1.0, 3.0, size=n_blobs)
    amps = rng.uniform(-amp, amp, size=n_blobs)
    drift = rng.uniform(-0.7, 0.7, size=(n_blobs, 3))
    for i in range(np_):
        for b in range(n_blobs):
            c = centres[b] + drift[b] * math.sin(2 * math.pi * i / max(np_, 1))
            r2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
            out[i] += amps[b] * np.exp(-0.5 * r2 / widths[b] ** 2)
    return out.astype(np.float32)
