"""The boundary from plain C: tests/c_abi_check.c links libtnlm.so and the
CUDA runtime, allocates device memory itself and calls the C ABI; its
checksums equal those of the Python binding on the same inputs."""
import os
import shutil
import subprocess

import numpy as np
import pytest
import torch

import paper_1201_2450_gb300 as tnlm

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _cuda_home():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def test_c_program_matches_binding(tmp_path):
    tnlm.build()
    lib = tnlm.library_path()
    cuda = _cuda_home()
    exe = str(tmp_path / "c_abi_check")
    libdir = os.path.join(cuda, "lib64")
    if not os.path.isdir(libdir):
        libdir = os.path.join(cuda, "lib")
    subprocess.run(["gcc", "-O1", "-std=c99", os.path.join(HERE, "c_abi_check.c"), "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(cuda, "include"), lib, "-L", libdir, "-lcudart", "-lm",
                    "-Wl,-rpath," + os.path.dirname(lib), "-Wl,-rpath," + libdir, "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    vals = {line.split()[0]: line.split()[1:] for line in out if line.strip()}

    angles = 2.0 * np.pi * np.arange(7) / 7.0 + 0.1
    desc = dict(nx=12, ny=10, nz=8, dx=1.0, dy=1.0, dz=1.0, cx=0.0, cy=0.0, cz=0.0, nu=24, nv=16, du=1.2, dv=1.2,
                u_off=0.0, v_off=0.0, sad=300.0, sdd=450.0, nviews=np.array([3, 4], np.int32), angles=angles)
    G = tnlm.Geometry(desc)
    vol = torch.from_numpy((np.arange(int(np.prod(G.vol_shape))) % 97).astype(np.float32)
                           * np.float32(1e-3)).reshape(G.vol_shape).cuda()
    proj = tnlm.tnlm_project(G, vol)
    assert float(vals["project"][0]) == pytest.approx(float(proj.double().sum()), rel=1e-12)
    bt = tnlm.tnlm_backproject(G, proj)
    assert float(vals["backproject"][0]) == pytest.approx(float(bt.double().sum()), rel=1e-12)
    f = torch.zeros(G.vol_shape, device="cuda")
    p = tnlm.Params(d=1, M=1, h=0.05, mu=1.0, tau=1e-4, n_outer=2, n_inner=1, clip_nonneg=1)
    _, rep = tnlm.tnlm_reconstruct(G, proj, f, p, report=True)
    r = [float(v) for v in vals["reconstruct"]]
    assert r[0] == pytest.approx(float(f.double().sum()), rel=1e-12)
    assert r[1:] == pytest.approx(list(rep.ravel()), rel=1e-12)
    assert vals["invalid"] == ["1", "invalid", "argument"]
