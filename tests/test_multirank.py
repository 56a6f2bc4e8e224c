"""The benchmark's multi-rank host logic on CPU (gloo, world size 2): the
barrier, the max-over-ranks timing and the whole-job aggregation of
independent per-rank reconstructions (no collective on the data path)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    assert (r, w, local) == (rank, world, rank)
    bench.barrier(w)
    ms = 100.0 + 50.0 * rank  # rank 1 is the slowest
    ms_max = bench.max_over_ranks(ms, w)
    out[rank] = (ms_max, bench.job_throughput(10, w, ms_max))
    dist.destroy_process_group()


def test_two_rank_timing_and_aggregation():
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1]
    ms_max, value = res[0]
    assert ms_max == 150.0
    assert value == pytest.approx(10 * 2 / 0.150)


def test_single_rank_defaults():
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_throughput(5, 1, 500.0) == pytest.approx(10.0)


def test_projection_nnz_counts_dense_matrix(ora):
    """The benchmark's algorithmic unit for the projector pair, nnz(P), equals
    the number of non-zeros of the oracle's dense P on a small geometry."""
    import numpy as np

    from paper_1201_2450_gb300 import synth
    g = synth.make_geometry(nx=6, ny=5, nz=4, dx=1.0, nu=12, nv=8, du=1.3, sad=40, sdd=60, n_phases=2,
                            views_per_phase=3, angle_offset=0.1)
    G = ora.Geometry(g)
    cols = []
    for ph in range(2):
        for v in range(6 * 5 * 4):
            e = np.zeros(G.vol_shape)
            e.reshape(2, -1)[ph, v] = 1.0
            cols.append(ora.project(G, e).ravel())
    P = np.stack(cols, 1)
    assert bench.projection_nnz(g, "cpu") == int((P > 1e-12).sum())
