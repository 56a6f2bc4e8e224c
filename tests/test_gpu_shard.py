"""The phase-sharded TNLM-R and TNLM-E on the GPU: two processes share the one
GPU (each owning a contiguous block of phases, running its own kernels) and
exchange their edge phases through gloo on the host between launches -- no
kernel waits for another.  The result equals the single-process
tnlm_reconstruct / tnlm_enhance bit for bit: every phase goes through the same
kernels with the same arithmetic, whichever process computes it."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import paper_1201_2450_gb300 as tnlm
from paper_1201_2450_gb300 import shard, synth

pytestmark = pytest.mark.gpu


def _geom(n_phases):
    return synth.make_geometry(nx=21, ny=18, nz=11, dx=1.5, nu=40, nv=20, du=1.4, sad=300, sdd=450,
                               n_phases=n_phases, views_per_phase=[5 + (i % 3) for i in range(n_phases)],
                               angle_offset=0.07)


def _recon_inputs(n_phases):
    g = _geom(n_phases)
    nviews = int(np.sum(g["nviews"]))
    y = synth.uniform((nviews, 20, 40), 500 + n_phases) * 0.3
    f0 = synth.smooth_volume((n_phases, 11, 18, 21), 510 + n_phases)
    return g, y, f0


def _enh_input(n_phases):
    shape = (n_phases, 12, 19, 23)
    return synth.smooth_volume(shape, 520 + n_phases) + synth.normal(shape, 521 + n_phases, 0.002)


CASES = {
    "R_np4": (4, dict(d=1, M=2, h=0.02, mu=0.8, tau=1e-4), 3, "R"),
    "R_np3_multisweep": (3, dict(d=2, M=1, h=0.03, mu=1.2, tau=5e-5, n_gj=2, gj_start=1), 2, "R"),
    "R_np2": (2, dict(d=1, M=3, h=0.02, mu=1.0, tau=1e-4), 2, "R"),
    "E_np5": (5, dict(d=2, M=3, h=0.04, mu=1.0, clip_nonneg=0), 3, "E"),
    "E_np2": (2, dict(d=1, M=2, h=0.02, mu=1.0, clip_nonneg=0), 2, "E"),
}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    for key, (n_phases, kw, n_outer, kind) in CASES.items():
        ex = shard.HaloExchange(rank, world, n_phases)
        a, b = ex.start, ex.stop
        p = tnlm.Params(n_outer=n_outer, **kw)
        if kind == "R":
            geom, y, f0 = _recon_inputs(n_phases)
            G = tnlm.Geometry(shard.local_geometry(geom, a, b))
            f = torch.from_numpy(np.ascontiguousarray(f0[a:b])).cuda()
            yl = torch.from_numpy(np.ascontiguousarray(shard.local_projections(geom, y, a, b))).cuda()
            rep = shard.reconstruct(ex, shard.GpuBackend(G, p), yl, f, p, n_outer, report=True)
            torch.cuda.synchronize()
            out[(key, rank)] = (f.cpu().numpy(), rep)
            G.close()
        else:
            g = torch.from_numpy(np.ascontiguousarray(_enh_input(n_phases)[a:b])).cuda()
            f = shard.enhance(ex, shard.GpuBackend(None, p), g, p, n_outer)
            torch.cuda.synchronize()
            out[(key, rank)] = (f.cpu().numpy(), None)
    dist.destroy_process_group()


def test_two_processes_equal_single_process_bitwise():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    tnlm.build()
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    torch.cuda.set_device(0)
    for key, (n_phases, kw, n_outer, kind) in CASES.items():
        p = tnlm.Params(n_outer=n_outer, **kw)
        if kind == "R":
            geom, y, f0 = _recon_inputs(n_phases)
            G = tnlm.Geometry(geom)
            f = torch.from_numpy(f0).cuda()
            _, rep = tnlm.tnlm_reconstruct(G, torch.from_numpy(y).cuda(), f, p, report=True)
            ref = f.cpu().numpy()
            G.close()
            np.testing.assert_allclose(res[(key, 0)][1], rep, rtol=1e-12)  # FP64 norms summed over ranks
        else:
            ref = tnlm.tnlm_enhance(torch.from_numpy(_enh_input(n_phases)).cuda(), p).cpu().numpy()
        got = np.concatenate([res[(key, r)][0] for r in range(2)])
        assert np.array_equal(got, ref), key
