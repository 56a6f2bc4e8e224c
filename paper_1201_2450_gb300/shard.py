"""Phase-sharded TNLM-R and TNLM-E across processes, one GPU each.

(P1) is uncoupled across phases (Sec. 2.3) and Eq. 8 couples phase i only to
its ring neighbours i +- 1 (periodic in phase, Sec. 2.1).  So each rank owns a
contiguous block of the N_p phases, runs (P1) and the Eq. 8 sweeps on its own
phases only, and before every sweep receives the two edge phases it needs from
its ring neighbours (the halo exchange): g^(k) once per TNLM-R iteration (and
the previous sweep's output when several sweeps run), f^(k) before every
TNLM-E sweep.  Ranks hold their phases in "extended" arrays of n_loc + 2
phases, [halo below, own phases, halo above]; the range sweep
(tnlm_gauss_jacobi_range) writes the own phases 1 .. n_loc, whose neighbours
are then all inside the array.  With N_p = 2 over two ranks both halos are the
other phase, the literal periodic reading used everywhere else.

The exchange is point-to-point (torch.distributed isend / irecv) between ring
neighbours; CUDA tensors are staged through host memory when the process group
is gloo.  The FP64 residual norms of (P1) are summed over ranks with one
all-reduce.  No step is computed here: the compute calls belong to a backend
(GpuBackend: the library's kernels; the tests also drive the same loops with
the FP64 oracle).
"""
from __future__ import annotations

import numpy as np
import torch


def phase_blocks(n_phases: int, world: int) -> list[tuple[int, int]]:
    """Contiguous blocks [start, stop) of the phases per rank; the first
    n_phases % world ranks own one phase more."""
    if world < 1 or n_phases < 2 or world > n_phases:
        raise ValueError(f"need 1 <= world <= n_phases and n_phases >= 2 (got {world}, {n_phases})")
    base, extra = divmod(n_phases, world)
    blocks, start = [], 0
    for r in range(world):
        stop = start + base + (1 if r < extra else 0)
        blocks.append((start, stop))
        start = stop
    return blocks


def halo_phases(n_phases: int, start: int, stop: int) -> tuple[int, int]:
    """The phases a block [start, stop) needs from outside: (start - 1) and stop, mod N_p."""
    return (start - 1) % n_phases, stop % n_phases


def owner(blocks: list[tuple[int, int]], phase: int) -> int:
    for r, (a, b) in enumerate(blocks):
        if a <= phase < b:
            return r
    raise ValueError(f"phase {phase} is owned by no rank")


def local_geometry(desc: dict, start: int, stop: int) -> dict:
    """The scan geometry of the phases [start, stop): the same volume and
    detector, those phases' views (phase-major angles)."""
    nviews = np.asarray(desc["nviews"], np.int32)
    off = np.concatenate([[0], np.cumsum(nviews)])
    out = dict(desc)
    out["nviews"] = nviews[start:stop].copy()
    out["angles"] = np.asarray(desc["angles"], np.float64)[off[start]:off[stop]].copy()
    return out


def local_projections(desc: dict, y, start: int, stop: int):
    """The rows of the phase-major projections y that belong to phases [start, stop)."""
    off = np.concatenate([[0], np.cumsum(np.asarray(desc["nviews"]))])
    return y[int(off[start]):int(off[stop])]


class HaloExchange:
    """Ring exchange of edge phases between neighbouring ranks.

    exchange(ext) fills ext[0] with the last phase of the rank below and
    ext[n_loc + 1] with the first phase of the rank above (ring order), from
    the own phases ext[1 .. n_loc].  Messages to one peer are posted in a
    fixed order (first own phase, then last) on both sides, so the exchange
    also pairs correctly with two ranks, where both neighbours are one rank,
    and on backends without message tags."""

    def __init__(self, rank: int, world: int, n_phases: int, dist=None):
        self.rank, self.world, self.n_phases = rank, world, n_phases
        self.blocks = phase_blocks(n_phases, world)
        self.start, self.stop = self.blocks[rank]
        self.n_loc = self.stop - self.start
        self.dist = dist
        if world > 1 and dist is None:
            import torch.distributed as dist_mod
            self.dist = dist_mod
        self.below = (rank - 1) % world
        self.above = (rank + 1) % world
        lo, hi = halo_phases(n_phases, self.start, self.stop)
        assert owner(self.blocks, lo) == self.below and owner(self.blocks, hi) == self.above
        self.messages = 0

    def _host_staged(self) -> bool:
        return self.world > 1 and self.dist.get_backend() != "nccl"

    def exchange(self, ext: torch.Tensor) -> None:
        n = self.n_loc
        if self.world == 1:  # the ring closes on this rank
            ext[0].copy_(ext[n])
            ext[n + 1].copy_(ext[1])
            return
        staged = self._host_staged() and ext.is_cuda
        first, last = ext[1], ext[n]
        if staged:
            first, last = first.cpu(), last.cpu()
            lo_buf, hi_buf = torch.empty_like(first), torch.empty_like(first)
        else:
            lo_buf, hi_buf = ext[0], ext[n + 1]
        d = self.dist
        ops = [d.P2POp(d.isend, first.contiguous(), self.below, tag=1),
               d.P2POp(d.isend, last.contiguous(), self.above, tag=2),
               d.P2POp(d.irecv, hi_buf, self.above, tag=1),
               d.P2POp(d.irecv, lo_buf, self.below, tag=2)]
        for req in d.batch_isend_irecv(ops):
            req.wait()
        if staged:
            ext[0].copy_(lo_buf)
            ext[n + 1].copy_(hi_buf)
        self.messages += 2

    def allreduce_sum(self, values: np.ndarray) -> np.ndarray:
        """FP64 sum over ranks (the residual norms of (P1))."""
        if self.world == 1:
            return values
        t = torch.as_tensor(values, dtype=torch.float64)
        if self.dist.get_backend() == "nccl":
            t = t.cuda()
        self.dist.all_reduce(t)
        return t.cpu().numpy()


class GpuBackend:
    """The compute steps of the sharded loops as calls of the library: (P1)
    on the rank's own phases (a geometry handle of those phases) and the range
    sweep on extended arrays."""

    def __init__(self, geom_local, params):
        from paper_1201_2450_gb300 import tnlm_gauss_jacobi_range, tnlm_p1
        self._p1, self._sweep = tnlm_p1, tnlm_gauss_jacobi_range
        self.geom, self.params = geom_local, params

    def p1(self, y, f_own, g_own, report: bool):
        return self._p1(self.geom, y, f_own, g_own, self.params, report=report)

    def sweep(self, wsrc, vals, g, out, n_loc, clip):
        p = self.params
        self._sweep(wsrc, vals, g, out, 1, n_loc, p.d, p.M, p.h, p.mu, clip)


def reconstruct(ex: HaloExchange, backend, y_local, f_own: torch.Tensor, params, n_outer: int,
                report: bool = False):
    """TNLM-R on this rank's phases, in place on f_own ([n_loc][nz][ny][nx]),
    in step with the other ranks; every iteration: (P1) on the own phases, halo
    exchange of g^(k), n_gj range sweeps (an exchange of the previous output
    before each further sweep), positivity after the last.  Returns the
    residual norms summed over ranks, [n_outer][n_inner], when report."""
    n = ex.n_loc
    shape = (n + 2,) + tuple(f_own.shape[1:])
    g_ext = torch.empty(shape, dtype=f_own.dtype, device=f_own.device)
    f_ext = torch.empty_like(g_ext)
    t_ext = torch.empty_like(g_ext)
    f_ext[1:n + 1].copy_(f_own)
    rows = []
    ngj = params.n_gj if params.n_gj > 0 else 1
    for _ in range(n_outer):
        rep = backend.p1(y_local, f_ext[1:n + 1], g_ext[1:n + 1], report)
        if report:
            rows.append(rep)
        ex.exchange(g_ext)
        vals = g_ext
        if params.gj_start:
            ex.exchange(f_ext)
            vals = f_ext
        for l in range(ngj):
            dst = f_ext if (ngj - 1 - l) % 2 == 0 else t_ext
            if dst is vals:
                dst = t_ext if vals is f_ext else f_ext
            backend.sweep(g_ext, vals, g_ext, dst, n, params.clip_nonneg if l == ngj - 1 else 0)
            if l < ngj - 1:
                ex.exchange(dst)
            vals = dst
        if vals is not f_ext:
            f_ext[1:n + 1].copy_(vals[1:n + 1])
    f_own.copy_(f_ext[1:n + 1])
    return ex.allreduce_sum(np.asarray(rows, np.float64)) if report else None


def enhance(ex: HaloExchange, backend, g_own: torch.Tensor, params, n_sweeps: int) -> torch.Tensor:
    """TNLM-E on this rank's phases: f^(0) = g, then n_sweeps of (halo
    exchange of f^(k), range sweep with fidelity image g).  Returns f_own."""
    n = ex.n_loc
    shape = (n + 2,) + tuple(g_own.shape[1:])
    g_ext = torch.zeros(shape, dtype=g_own.dtype, device=g_own.device)
    g_ext[1:n + 1].copy_(g_own)
    a = g_ext.clone()
    b = torch.empty_like(a)
    for _ in range(n_sweeps):
        ex.exchange(a)
        backend.sweep(a, a, g_ext, b, n, params.clip_nonneg)
        a, b = b, a
    return a[1:n + 1].clone()
