"""The phase-sharded form of TNLM-R and TNLM-E on CPU: the partition and halo
bookkeeping, and the sharded loops run as two gloo ranks with the FP64 oracle
as the compute backend, equal bit for bit to the same loops on one rank and to
the oracle's own TNLM-E (uneven blocks, N_p = 2 over two ranks, the ring wrap
at both ends)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1201_2450_gb300 import shard, synth


def test_phase_blocks_and_halos():
    assert shard.phase_blocks(10, 1) == [(0, 10)]
    assert shard.phase_blocks(10, 4) == [(0, 3), (3, 6), (6, 8), (8, 10)]
    assert shard.phase_blocks(3, 2) == [(0, 2), (2, 3)]
    assert shard.phase_blocks(2, 2) == [(0, 1), (1, 2)]
    for n, w in [(10, 3), (7, 7), (5, 2), (2, 2)]:
        b = shard.phase_blocks(n, w)
        assert b[0][0] == 0 and b[-1][1] == n
        assert all(b[r][1] == b[r + 1][0] for r in range(w - 1))
        assert max(s - a for a, s in b) - min(s - a for a, s in b) <= 1
        for r, (a, s) in enumerate(b):
            lo, hi = shard.halo_phases(n, a, s)
            assert shard.owner(b, lo) == (r - 1) % w and shard.owner(b, hi) == (r + 1) % w
    assert shard.halo_phases(10, 0, 3) == (9, 3)    # the ring wraps below phase 0
    assert shard.halo_phases(10, 8, 10) == (7, 0)   # and above phase N_p - 1
    assert shard.halo_phases(2, 0, 1) == (1, 1)     # N_p = 2: both halos are the other phase
    with pytest.raises(ValueError):
        shard.phase_blocks(3, 4)
    with pytest.raises(ValueError):
        shard.phase_blocks(1, 1)


def test_local_geometry_and_projections():
    g = synth.make_geometry(nx=8, ny=8, nz=4, dx=1.0, nu=10, nv=6, du=1.0, n_phases=3, views_per_phase=[2, 3, 4])
    lg = shard.local_geometry(g, 1, 3)
    assert list(lg["nviews"]) == [3, 4]
    assert np.array_equal(lg["angles"], np.asarray(g["angles"])[2:9])
    y = np.arange(9 * 6 * 10).reshape(9, 6, 10)
    assert np.array_equal(shard.local_projections(g, y, 1, 3), y[2:9])
    assert np.array_equal(shard.local_projections(g, y, 0, 1), y[0:2])


class OracleBackend:
    """The sharded loops' compute steps by the FP64 oracle: the sweep of the
    extended array (every phase, with the ring wrap; only the own phases
    1 .. n_loc are kept, whose neighbours lie inside the array), and (P1) as
    gradient steps g <- g - tau P^T (P g - y) on the rank's own phases."""

    def __init__(self, ora, geom_local, params):
        self.ora, self.params = ora, params
        self.OG = ora.Geometry(geom_local)

    def p1(self, y, f_own, g_own, report):
        p, o = self.params, self.ora
        g = f_own.numpy().copy()
        rep = []
        for _ in range(p.n_inner):
            r = o.project(self.OG, g) - y
            rep.append(float((r * r).sum()))
            g = g - p.tau * o.backproject(self.OG, r)
        g_own.copy_(torch.from_numpy(g))
        return np.array(rep) if report else None

    def sweep(self, wsrc, vals, g, out, n_loc, clip):
        p = self.params
        full = self.ora.gj_sweep(wsrc.numpy(), vals.numpy(), g.numpy(), p.d, p.M, p.h, p.mu, clip)
        out[1:n_loc + 1].copy_(torch.from_numpy(full[1:n_loc + 1]))


class P:
    def __init__(self, **kw):
        self.d, self.M, self.h, self.mu, self.tau = 1, 1, 0.05, 0.9, 3e-3
        self.n_inner, self.n_gj, self.gj_start, self.clip_nonneg = 1, 1, 0, 1
        self.__dict__.update(kw)


def _problem(n_phases):
    geom = synth.make_geometry(nx=7, ny=6, nz=5, dx=1.0, nu=12, nv=8, du=1.1, sad=60, sdd=90, n_phases=n_phases,
                               views_per_phase=[2 + (i % 2) for i in range(n_phases)], angle_offset=0.05)
    f0 = synth.smooth_volume((n_phases, 5, 6, 7), 400 + n_phases)
    y = synth.uniform((sum(geom["nviews"]), 8, 12), 410 + n_phases) * 0.2
    return geom, f0.astype(np.float64), y.astype(np.float64)


def _run(ora, rank, world, n_phases, params, n_outer, kind, dist_mod=None):
    geom, f0, y = _problem(n_phases)
    ex = shard.HaloExchange(rank, world, n_phases, dist=dist_mod)
    a, b = ex.start, ex.stop
    be = OracleBackend(ora, shard.local_geometry(geom, a, b), params)
    if kind == "R":
        f = torch.from_numpy(f0[a:b].copy())
        rep = shard.reconstruct(ex, be, shard.local_projections(geom, y, a, b), f, params, n_outer, report=True)
        return f.numpy(), rep, ex.messages
    g = torch.from_numpy(f0[a:b].copy())
    return shard.enhance(ex, be, g, params, n_outer).numpy(), None, ex.messages


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, cases, out):
    import oracle as ora
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    for key, (n_phases, kw, n_outer, kind) in cases.items():
        out[(key, rank)] = _run(ora, rank, world, n_phases, P(**kw), n_outer, kind, dist)
    dist.destroy_process_group()


CASES = {
    "R_np2": (2, {}, 2, "R"),                                      # one phase per rank, both halos the other
    "R_np3_uneven_multisweep": (3, {"n_gj": 2, "gj_start": 1}, 2, "R"),  # blocks 2 + 1, exchanges per sweep
    "R_np5_inner2": (5, {"n_inner": 2, "clip_nonneg": 0}, 2, "R"),
    "E_np5": (5, {"clip_nonneg": 0}, 3, "E"),
    "E_np2": (2, {"clip_nonneg": 0}, 2, "E"),
}


def test_two_gloo_ranks_equal_one_rank(ora):
    ora.build()
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, CASES, out), nprocs=2, join=True)
        res = dict(out)
    for key, (n_phases, kw, n_outer, kind) in CASES.items():
        single, rep1, _ = _run(ora, 0, 1, n_phases, P(**kw), n_outer, kind)
        blocks = shard.phase_blocks(n_phases, 2)
        got = np.concatenate([res[(key, r)][0] for r in range(2)])
        assert got.shape == single.shape
        assert np.array_equal(got, single), key       # the same arithmetic per phase, bit for bit
        assert res[(key, 0)][2] == res[(key, 1)][2] > 0  # every rank took part in every exchange
        if kind == "R":
            np.testing.assert_allclose(res[(key, 0)][1], rep1, rtol=1e-13)  # residuals summed over ranks
            assert np.array_equal(res[(key, 0)][1], res[(key, 1)][1])
        assert [b - a for a, b in blocks] == [res[(key, r)][0].shape[0] for r in range(2)]


def test_single_rank_loops_equal_the_oracle(ora):
    """The loops on one rank (the ring closed on itself) reproduce the
    oracle's TNLM-E exactly and its TNLM-R to rounding (its (P1) is composed
    from the oracle's P and P^T here)."""
    ora.build()
    f, _, _ = _run(ora, 0, 1, 5, P(clip_nonneg=0), 3, "E")
    geom, f0, y = _problem(5)
    assert np.array_equal(f, ora.enhance(f0, 1, 1, 0.05, 0.9, 3))
    p = P(n_gj=2, gj_start=1)
    f, rep, _ = _run(ora, 0, 1, 3, p, 2, "R")
    geom, f0, y = _problem(3)
    ref, rep_ref = ora.reconstruct(ora.Geometry(geom), y, f0, p.tau, p.d, p.M, p.h, p.mu, 2, n_inner=1, clip=1,
                                   gj_start=1, n_gj=2, with_report=True)
    np.testing.assert_allclose(f, ref, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(rep, rep_ref, rtol=1e-12)
