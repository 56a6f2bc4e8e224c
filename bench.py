#!/usr/bin/env python3
"""Benchmark of the TNLM 4D-CBCT forward-backward-splitting hot path on GB300.

Workload (the NCAT-shaped reconstruction): 10 phases, 256 x 256 x 64 volume
at 2 mm, 36 views per phase (360 over one rotation, phase-interleaved) on a
512 x 384 detector at 0.78 mm, SAD 1000 / SDD 1500 mm, patch 3^3 (d = 1),
search window 7^3 (M = 3), h = 0.02, mu = 1.  Inputs are synthetic: a seeded
thorax phantom, analytic line integrals, Poisson noise at I0 = 5e4.

One step = one FBS iteration of TNLM-R through tnlm_reconstruct: forward
projection + residual of every phase, voxel-driven transpose + gradient
step, fused weights + Gauss-Jacobi sweep + positivity.  Inputs (y: 283 MB,
f: 168 MB) exceed the 129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank reconstructs its own problem (independent 4D
reconstructions, weak scaling, no collective on the data path); rank 0
prints one JSON line.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FBS iterations/s and TNLM voxel-updates/s on 1 GB300; % HBM roofline vs FP32"
UNIT = "FBS iterations/s"
WORKLOAD = ("NCAT-shaped 4D TNLM-R FP32: 10 phases x 256x256x64 @ 2 mm, 36 views/phase on 512x384 @ 0.78 mm, "
            "SAD 1000 / SDD 1500, patch 3^3, window 7^3, h 0.02, mu 1")

# ncu DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of
# each kernel on this workload, with the SHA-256 of the kernel source it was
# measured on; a changed source invalidates the figure (reported as null).
NCU_TRAFFIC = {
    # single-kernel captures on the 6-phase case of this workload, scaled by 10/6 to its 10 phases; the
    # projector stage is the bricked copy plus the table walk, the transpose stage the column scan plus the bands
    "k_forward": {"bytes_per_launch": int((100.727808e6 + 48.609024e6 + 606.395392e6 + 165.109504e6) * 10 / 6),
                  "source_sha": "4ee81dbf075d39bb"},
    "k_backproject": {"bytes_per_launch": int((169.919488e6 + 284.322560e6 + 556.931328e6 + 93.128448e6) * 10 / 6),
                      "source_sha": "5aa935fcb93c583b"},
    "k_sweep": {"bytes_per_launch": int((162.544640e6 + 83.844608e6) * 10 / 6), "source_sha": "aa475743b3412a05"},
}


def _src_sha(fname: str) -> str:
    p = os.path.join(ROOT, "paper_1201_2450_gb300", "csrc", fname)
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


KERNEL_SRC = {"k_forward": "projector.cu", "k_backproject": "transpose.cu", "k_sweep": "sweep_box.cuh"}


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        d["_source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0, "_source": "fallback"}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if "Active" in r[5 + k] and "Not" not in r[5 + k]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    """Slowest rank's value (the job ends when the last rank does)."""
    if world == 1:
        return x
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(steps: int, world: int, ms_max: float) -> float:
    """Whole-job FBS iterations/s: every rank runs `steps` iterations of its own
    reconstruction; the job takes the slowest rank's time."""
    return steps * world / (ms_max / 1e3)


# ---------------------------------------------------------------------------
# algorithmic work and bytes per launch: each kernel's unit count times its per-unit bytes or operations
# ---------------------------------------------------------------------------

def algorithmic_bytes(cfg, n_views_total):
    npz = cfg.n_phases * cfg.vol[0] * cfg.vol[1] * cfg.vol[2]
    npix = n_views_total * cfg.det[0] * cfg.det[1]
    return {
        "k_forward": 4 * npz + 4 * npix + 4 * npix,     # read f, read y, write scaled residual
        "k_backproject": 4 * npix + 4 * npz + 4 * npz,  # read residual, read f, write g
        "k_sweep": 4 * npz + 4 * npz,                   # read g (weights, values, fidelity), write f
    }


def projection_nnz(desc: dict, device="cuda") -> int:
    """Non-zeros of P: the number of (ray, cell) pairs with a positive chord,
    i.e. cells crossed per ray = 1 + sum over axes of |exit cell - entry cell|
    (FP64, counted view by view on the device)."""
    return projection_counts(desc, device)[0]


# FP32 operations of the projector's slab walk, counted from its source (an FMA counts 2): per
# dominant-axis slab 12 (slab end, crossing test and select, two segment lengths and FMAs, the next
# plane by one FMA), per in-plane (b) crossing 3 more, per z (c) crossing 7 (its segment and the next
# z plane); so per ray 12 (1 + |da|) + 3 |db| + 7 |dc| with da, db, dc the cell steps along each axis.
K1_FLOP_SLAB, K1_FLOP_B, K1_FLOP_C = 12, 3, 7
# FP32 operations of the table walk (the default projector), counted from its source: per xy-table
# entry 3 (its segment length and FMA; only a row's last entry is clamped to its exit), per z crossing
# 6 (its segment length and FMA, the next z plane by an add and one FMA); so per ray
# 3 (1 + |dx| + |dy|) + 6 |dz|.  The tables themselves are built once per geometry, not per launch.
K1_TAB_FLOP_ENTRY, K1_TAB_FLOP_C = 3, 6
# FP32 operations of the band transpose per non-zero of P, counted from its source on this geometry
# (an FMA counts 2, a min/max or a conversion 1): per (column of 8 cells, view, pixel column) 38 for
# the chord (two slab tests) and the row-map slopes, 12 for the chord midpoint, the first boundary
# and its row images, then 30 per cell boundary (the boundary height, its two row images with their
# margins, the band row's split and its two accumulations, the prefix difference of the full rows),
# 320 in all, plus ~13 for the column's footprint per view shared by its ~3.5 pixel columns, over
# the ~38 (ray, cell) pairs that chord serves (about 4.8 detector rows per 2 mm cell).
K2_FLOP_PER_NNZ = 8.5


def projection_counts(desc: dict, device="cuda") -> tuple[int, int, int]:
    """(nnz(P), FP32 operations of the slab walk, of the table walk), exact
    per ray from the entry and exit cells along each axis; the slab walk's
    dominant axis is x or y (the steeper of the two, z when steeper still),
    as in the kernel."""
    nu, nv = desc["nu"], desc["nv"]
    dev = torch.device(device)
    u = (torch.arange(nu, device=dev, dtype=torch.float64) - 0.5 * (nu - 1)) * desc["du"] + desc["u_off"]
    v = (torch.arange(nv, device=dev, dtype=torch.float64) - 0.5 * (nv - 1)) * desc["dv"] + desc["v_off"]
    V, U = torch.meshgrid(v, u, indexing="ij")
    flops = flops_tab = 0
    n = [desc["nx"], desc["ny"], desc["nz"]]
    w = [desc["dx"], desc["dy"], desc["dz"]]
    b0 = [desc["cx"] - 0.5 * n[0] * w[0], desc["cy"] - 0.5 * n[1] * w[1], desc["cz"] - 0.5 * n[2] * w[2]]
    total = 0
    for th in desc["angles"]:
        c, s_ = float(np.cos(th)), float(np.sin(th))
        src = [desc["sad"] * c, desc["sad"] * s_, 0.0]
        pix = [(desc["sad"] - desc["sdd"]) * c - U * s_, (desc["sad"] - desc["sdd"]) * s_ + U * c, V]
        d = [pix[k] - src[k] for k in range(3)]
        amin = torch.zeros_like(U)
        amax = torch.ones_like(U)
        for k in range(3):
            a0 = (b0[k] - src[k]) / d[k]
            a1 = (b0[k] + n[k] * w[k] - src[k]) / d[k]
            amin = torch.maximum(amin, torch.minimum(a0, a1))
            amax = torch.minimum(amax, torch.maximum(a0, a1))
        hit = amin < amax
        eps = 1e-9
        cnt = torch.ones_like(U)
        steps = []
        for k in range(3):
            ce = torch.floor((src[k] + (amin + eps) * d[k] - b0[k]) / w[k])
            cx_ = torch.floor((src[k] + (amax - eps) * d[k] - b0[k]) / w[k])
            steps.append(torch.abs(cx_ - ce))
            cnt += steps[-1]
        g = [torch.abs(d[k]) / w[k] for k in range(3)]
        zdom = (g[2] > g[0]) & (g[2] > g[1])
        xa = ~zdom & (g[0] >= g[1])
        sa = torch.where(zdom, steps[2], torch.where(xa, steps[0], steps[1]))
        sb = torch.where(xa, steps[1], steps[0])
        sc = torch.where(zdom, steps[1], steps[2])
        fl = K1_FLOP_SLAB * (1 + sa) + K1_FLOP_B * sb + K1_FLOP_C * sc
        ft = K1_TAB_FLOP_ENTRY * (1 + steps[0] + steps[1]) + K1_TAB_FLOP_C * steps[2]
        zero = torch.zeros_like(cnt)
        total += int(torch.where(hit, cnt, zero).sum().item())
        flops += int(torch.where(hit, fl, zero).sum().item())
        flops_tab += int(torch.where(hit, ft, zero).sum().item())
    return total, flops, flops_tab


# FP32 operations per pair evaluation of the sweep (the hot-path analysis's per-unit figure):
# 3*3*(2d+1) for the box-sum patch distance plus 8 for the weight and the two accumulations
# (one exp besides).


def sweep_ops_per_pair(d: int) -> int:
    return 9 * (2 * d + 1) + 8


def measure_compute_peaks(tnlm, stream, gpu_index: int) -> dict:
    """The compute roofline's denominators measured on this GPU: FP32 FMA
    (scalar FFMA and packed FP32x2), and ex2, each probe launched alone on
    8 blocks of 256 threads per SM (8 independent chains per thread) and timed
    with CUDA events on `stream` (best of 5 after 2 warm-ups), while the SM
    clock is sampled; the SM count is the device's own."""
    props = torch.cuda.get_device_properties(gpu_index)
    sms = int(props.multi_processor_count)
    blocks = 8 * sms
    sink = torch.zeros(1, device="cuda")
    res = {"sms": sms, "device": props.name}
    sampler = ClockSampler(gpu_index)
    sampler.start()
    for kind, name, iters in ((0, "ffma", 40000), (1, "ffma2", 20000), (2, "ex2", 4000)):
        ms = []
        ops = 0.0
        for rep in range(7):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ops = tnlm.tnlm_peak_probe(kind, blocks, iters, sink, stream=stream)
            e1.record(stream)
            e1.synchronize()
            if rep >= 2:
                ms.append(e0.elapsed_time(e1))
        rate = ops / (min(ms) / 1e3)
        if kind < 2:
            res[f"{name}_tflops"] = round(rate / 1e12, 3)
        else:
            res["ex2_per_s"] = float(f"{rate:.4g}")
    res["clocks"] = sampler.stop()
    res["fp32_tflops"] = max(res["ffma_tflops"], res["ffma2_tflops"])
    return res


def sweep_pairs(cfg):
    """Pair evaluations of one sweep: every voxel, both directions, every
    window offset that stays inside the volume."""
    nx, ny, nz = cfg.vol
    M = cfg.M

    def valid(n):
        return sum(min(n - 1, i + M) - max(0, i - M) + 1 for i in range(n))

    return 2 * cfg.n_phases * valid(nx) * valid(ny) * valid(nz)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args, rank, world, local):
    import paper_1201_2450_gb300 as tnlm
    from paper_1201_2450_gb300 import synth

    torch.cuda.set_device(local)
    tnlm.build()
    cfg = synth.C2
    if args.phases != cfg.n_phases:  # smaller case of the same kernels (profiling captures)
        cfg = dataclasses.replace(cfg, n_phases=args.phases)
    pb = synth.recon_problem(cfg, device="cuda")  # same seeded problem on every rank
    geom = tnlm.Geometry(pb.geom)
    y = pb.y.contiguous()
    x0 = torch.from_numpy(synth.uniform(geom.vol_shape, 2024)).cuda()
    L = tnlm.tnlm_operator_norm(geom, x0, args.power_iters)
    tau = 1.0 / L
    params = tnlm.Params(d=cfg.d, M=cfg.M, h=cfg.h, mu=cfg.mu, tau=tau, n_outer=1, n_inner=1, clip_nonneg=1)
    # storage of y, f and the iteration's images: FP32 (the benchmark), or BF16 / FP16 with FP32 arithmetic
    sdtype, recon = {"fp32": (torch.float32, tnlm.tnlm_reconstruct), "bf16": (torch.bfloat16, tnlm.tnlm_reconstruct_bf16),
                     "fp16": (torch.float16, tnlm.tnlm_reconstruct_fp16)}[args.storage]
    ys = y.to(sdtype).contiguous()
    f = torch.zeros(geom.vol_shape, device="cuda", dtype=sdtype)
    stream = torch.cuda.current_stream()
    # launch shapes: timed once on this problem before the run (results do not depend on them)
    shapes = None if args.no_autotune else tnlm.tnlm_autotune(geom, params)

    for _ in range(args.warmup):
        recon(geom, ys, f, params)
    torch.cuda.synchronize()

    geom.set_stage_timing(True)
    sampler = ClockSampler(local)
    sampler.start()
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        recon(geom, ys, f, params)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    ms_total = e0.elapsed_time(e1)
    stage_ms, stage_n = geom.stage_timing()
    geom.set_stage_timing(False)
    ms_max = max_over_ranks(ms_total, world)
    value = job_throughput(args.steps, world, ms_max)

    # end to end through the public API with host buffers
    y_host = y.cpu().pin_memory()
    f_host = torch.zeros(geom.vol_shape).pin_memory()
    y_dev = torch.empty_like(y)
    f_dev = torch.empty(geom.vol_shape, device="cuda")
    tnlm.reconstruct_host(geom, y_host, f_host, params, y_dev, f_dev)  # warm
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    h2d = d2h = 0
    e_steps = max(1, args.steps)  # as many steps as the device-timed loop
    for _ in range(e_steps):
        h2d, d2h = tnlm.reconstruct_host(geom, y_host, f_host, params, y_dev, f_dev)
        stream.synchronize()  # the host reads this step's result before the next step starts
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e_value = e_steps * world / e2e_s

    variants = {} if args.no_variants else measure_variants(tnlm, synth, geom, y, stream, params)

    peaks = measured_peaks()
    cpk = measure_compute_peaks(tnlm, stream, local)
    names = ["k_forward", "k_backproject", "k_sweep"]
    per_launch_ms = {n: stage_ms[k] / max(stage_n[k], 1) for k, n in enumerate(names)}
    abytes = algorithmic_bytes(cfg, geom.proj_shape[0])
    hbm = {}
    for n in names:
        gbs = abytes[n] / (per_launch_ms[n] / 1e3) / 1e9
        hbm[n] = {"ms_per_launch": round(per_launch_ms[n], 4), "algorithmic_bytes": abytes[n],
                  "achieved_gbs": round(gbs, 2), "frac_of_hbm": round(gbs / peaks["hbm_gbs"], 5)}
    dom = max(names, key=lambda n: per_launch_ms[n])
    traffic = None
    t = NCU_TRAFFIC.get(dom)
    if t and t.get("source_sha") == _src_sha(KERNEL_SRC[dom]) and cfg.n_phases == 10:
        traffic = t["bytes_per_launch"]
    # the three kernels are bound by FP32 / integer issue, not HBM: roofline against the FP32 peak
    nnz, k1_slab, k1_tab = projection_counts(pb.geom)
    in_use = tnlm.tnlm_get_launch_shapes(geom)
    k1_table = in_use["projector_rows"] > 100
    work = {"k_forward": k1_tab if k1_table else k1_slab, "k_backproject": K2_FLOP_PER_NNZ * nnz,
            "k_sweep": sweep_ops_per_pair(cfg.d) * sweep_pairs(cfg)}
    peak_t = cpk["fp32_tflops"]
    alu = {n: {"algorithmic_tflop": round(work[n] / 1e12, 4),
               "achieved_tflops": round(work[n] / (per_launch_ms[n] / 1e3) / 1e12, 3),
               "frac_of_fp32_peak": round(work[n] / (per_launch_ms[n] / 1e3) / 1e12 / peak_t, 4)} for n in names}
    roofline = {"bound": "alu", "kernel": dom, "achieved": alu[dom]["achieved_tflops"], "peak": round(peak_t, 2),
                "unit": "TFLOP/s", "frac": alu[dom]["frac_of_fp32_peak"], "traffic": traffic,
                "peak_source": f"measured FP32 FMA throughput of this GPU ({cpk['sms']} SMs; FFMA "
                               f"{cpk['ffma_tflops']} and packed FFMA2 {cpk['ffma2_tflops']} TFLOP/s, the larger "
                               f"taken; SM clock median {cpk['clocks'].get('sm_mhz')} MHz during the probes)",
                "work": f"{work[dom]:.4g} FP32 ops per launch (nnz(P) = {nnz:.4g})",
                "hbm_frac": hbm[dom]["frac_of_hbm"]}
    nvox_upd = cfg.n_phases * cfg.vol[0] * cfg.vol[1] * cfg.vol[2]
    sweep_s = per_launch_ms["k_sweep"] / 1e3
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "phases": cfg.n_phases, "volume": list(cfg.vol), "voxel_mm": cfg.voxel_mm,
                   "views_per_phase": cfg.views_per_phase, "detector": list(cfg.det), "pixel_mm": cfg.pixel_mm,
                   "d": cfg.d, "M": cfg.M, "h": cfg.h, "mu": cfg.mu, "tau": tau, "n_inner": 1,
                   "step": "one FBS iteration (projection+residual, transpose+gradient step, weights+Gauss-Jacobi+clip)",
                   "l2": "inputs larger than L2 (y 283 MB, f 168 MB), no flush",
                   "parallelism": f"replicas x{world} (independent reconstructions)",
                   "launch_shapes": dict(in_use, sweep_shape=shapes["sweep_shape"] if shapes else "default",
                                         projector_walker="table" if k1_table else "slab",
                                         autotuned=shapes is not None)},
        "tnlm_voxel_updates_per_s": round(nvox_upd / sweep_s, 1),
        "projector_segments_per_s": round(nnz / (per_launch_ms["k_forward"] / 1e3), 1),
        "transpose_segments_per_s": round(nnz / (per_launch_ms["k_backproject"] / 1e3), 1),
        "tnlm_pair_evals_per_s": round(sweep_pairs(cfg) / sweep_s, 1),
        "stage_ms_per_launch": {n: round(per_launch_ms[n], 4) for n in names},
        "hbm": hbm,
        "alu": alu,
        "compute_peaks": cpk,
        "roofline": roofline,
        "clocks": clocks,
        # per step: the projector stage (k_brick + k_forward_tab, or k_forward alone), the transpose stage
        # (k_colscan + k_backproject_bands on this workload), k_sweep_box
        "gpu_launches": int(stage_n[0] * (2 if k1_table else 1) + 2 * stage_n[1] + stage_n[2]),
        "e2e": {"value": round(e2e_value, 4), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "variants": variants,
    }
    if args.storage != "fp32":
        line["config"]["storage"] = f"{args.storage} storage of y, f and the iteration images, FP32 arithmetic"
        line["config"]["workload"] += f" [{args.storage} storage]"
    if args.phases != 10:
        line["config"]["workload"] += f" [reduced to {args.phases} phases]"
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample(cfg, pb)
    return line


def _time_ms(fn, stream, reps=3):
    """Median CUDA-event time of fn() on `stream` over reps runs (after one warm-up)."""
    fn()
    out = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        out.append(a.elapsed_time(b))
    return statistics.median(out)


def measure_variants(tnlm, synth, geom, y, stream, params) -> dict:
    """Steps either side of the FBS iteration and the enhancement workload:
    FDK of all phases, one CGLS iteration of (P1), and TNLM-E on
    10 x 512x512x128 (d = 2, M = 3, h = 0.04) in FP32."""
    out = {}
    vol = torch.empty(geom.vol_shape, device="cuda")
    out["fdk_ms"] = round(_time_ms(lambda: tnlm.tnlm_fdk(geom, y, vol), stream), 3)
    x = torch.zeros(geom.vol_shape, device="cuda")
    n_it = 3
    ms = _time_ms(lambda: tnlm.tnlm_cgls(geom, y, x, n_it), stream)
    x0 = torch.zeros(geom.vol_shape, device="cuda")
    ms0 = _time_ms(lambda: tnlm.tnlm_cgls(geom, y, x0, 0), stream)
    out["cgls_ms_per_iteration"] = round((ms - ms0) / n_it, 3)
    out["cgls_setup_ms"] = round(ms0, 3)
    # TNLM-R with BF16 storage on the same workload (3 iterations from 0 against the FP32 result)
    p3 = tnlm.Params(d=params.d, M=params.M, h=params.h, mu=params.mu, tau=params.tau, n_outer=3, clip_nonneg=1)
    y16 = y.bfloat16()
    f16 = torch.zeros(geom.vol_shape, device="cuda", dtype=torch.bfloat16)
    f32 = torch.zeros(geom.vol_shape, device="cuda")

    def r16():
        f16.zero_()
        tnlm.tnlm_reconstruct_bf16(geom, y16, f16, p3)

    def r32():
        f32.zero_()
        tnlm.tnlm_reconstruct(geom, y, f32, p3)

    yh = y.half()
    fh = torch.zeros(geom.vol_shape, device="cuda", dtype=torch.float16)

    def rh():
        fh.zero_()
        tnlm.tnlm_reconstruct_fp16(geom, yh, fh, p3)

    ms16 = _time_ms(r16, stream)
    msh = _time_ms(rh, stream)
    ms32 = _time_ms(r32, stream)

    def rel(a):
        return float(f"{float(torch.linalg.vector_norm((a.float() - f32).double()) / torch.linalg.vector_norm(f32.double())):.3e}")

    out["bf16_recon_ms_per_iteration"] = round(ms16 / 3, 3)
    out["fp16_recon_ms_per_iteration"] = round(msh / 3, 3)
    out["fp32_recon_ms_per_iteration_same_run"] = round(ms32 / 3, 3)
    out["bf16_recon_rel_l2_vs_fp32_3_iterations"] = rel(f16)
    out["fp16_recon_rel_l2_vs_fp32_3_iterations"] = rel(fh)
    del y16, f16, f32, yh, fh
    c3 = synth.C3
    g, _ = synth.enhance_input(c3, device="cuda")
    f = torch.empty_like(g)
    p = tnlm.Params(d=c3.d, M=c3.M, h=c3.h, mu=c3.mu, n_outer=1, clip_nonneg=0)
    out["tnlm_e_sweep_shape"] = tnlm.tnlm_autotune_sweep(tuple(g.shape), c3.d, c3.M, c3.h)
    out["tnlm_e_bf16_sweep_shape"] = tnlm.tnlm_autotune_sweep(tuple(g.shape), c3.d, c3.M, c3.h, bf16=True)
    sweep_ms = _time_ms(lambda: tnlm.tnlm_enhance(g, p, out=f), stream, reps=2)
    nvox = c3.n_phases * c3.vol[0] * c3.vol[1] * c3.vol[2]
    out["tnlm_e_workload"] = "TNLM-E FP32 10 x 512x512x128, patch 5^3, window 7^3, h 0.04, mu 1"
    out["tnlm_e_ms_per_sweep"] = round(sweep_ms, 3)
    out["tnlm_e_voxel_updates_per_s"] = round(nvox / (sweep_ms / 1e3), 1)
    out["tnlm_e_pair_evals_per_s"] = round(sweep_pairs(c3) / (sweep_ms / 1e3), 1)
    gb = g.to(torch.bfloat16)
    fb = torch.empty_like(gb)
    bf_ms = _time_ms(lambda: tnlm.tnlm_enhance_bf16(gb, p, out=fb), stream, reps=2)
    out["tnlm_e_bf16_ms_per_sweep"] = round(bf_ms, 3)
    out["tnlm_e_bf16_voxel_updates_per_s"] = round(nvox / (bf_ms / 1e3), 1)
    out["tnlm_e_fp16_sweep_shape"] = tnlm.tnlm_autotune_sweep(tuple(g.shape), c3.d, c3.M, c3.h, fp16=True)
    gh = g.half()
    fhh = torch.empty_like(gh)
    h_ms = _time_ms(lambda: tnlm.tnlm_enhance_fp16(gh, p, out=fhh), stream, reps=2)
    out["tnlm_e_fp16_ms_per_sweep"] = round(h_ms, 3)
    out["tnlm_e_fp16_voxel_updates_per_s"] = round(nvox / (h_ms / 1e3), 1)
    del g, f, gb, fb, gh, fhh
    torch.cuda.empty_cache()
    # differentiable total energy (frozen weights) on 10 x 128^3, 40 views x 256x192
    c4 = synth.C4
    pb4 = synth.recon_problem(c4, device="cuda")
    g4 = tnlm.Geometry(pb4.geom)
    f4 = (pb4.truth + 0.001).contiguous()
    grad4 = torch.empty_like(f4)
    p4 = tnlm.Params(d=c4.d, M=c4.M, h=c4.h, mu=c4.mu)
    out["energy_grad_workload"] = "E(f) and grad E, 10 x 128^3 at 2 mm, 40 views x 256x192, patch 3^3, window 5^3"
    out["energy_grad_ms"] = round(_time_ms(lambda: tnlm.tnlm_energy_grad(g4, pb4.y, f4, pb4.truth, p4, grad=grad4),
                                           stream), 3)
    y16, f16, a16 = pb4.y.bfloat16(), f4.bfloat16(), pb4.truth.bfloat16()
    out["energy_grad_bf16_ms"] = round(_time_ms(lambda: tnlm.tnlm_energy_grad_bf16(g4, y16, f16, a16, p4, grad=grad4),
                                                stream), 3)
    del y16, f16, a16
    ga4 = torch.empty_like(f4)
    out["energy_grad_weights_ms"] = round(_time_ms(
        lambda: tnlm.tnlm_energy_grad_weights(f4, pb4.truth, c4.d, c4.M, c4.h, grad_a=ga4), stream), 3)
    del ga4
    g4.close()
    del pb4, f4, grad4
    torch.cuda.empty_cache()
    out.update(measure_batch(tnlm, synth, stream))
    out.update(measure_c1_latency(tnlm, synth, stream))
    return out


def measure_c1_latency(tnlm, synth, stream) -> dict:
    """The small plain TNLM-R problem (4 x 32^3, 20 views x 64x48, patch 3^3,
    window 5^3, 5 iterations) is launch-bound: ms per FBS iteration through
    tnlm_reconstruct (one launch sequence per iteration) and through the
    captured-graph form (tnlm_reconstruct_batch with one problem)."""
    c1 = synth.C1
    pb = synth.recon_problem(c1, device="cuda")
    g = tnlm.Geometry(pb.geom)
    p = tnlm.Params(d=c1.d, M=c1.M, h=c1.h, mu=c1.mu, tau=1e-4, n_outer=c1.n_outer)
    f = torch.zeros(g.vol_shape, device="cuda")
    plain = _time_ms(lambda: tnlm.tnlm_reconstruct(g, pb.y, f, p), stream, reps=5)
    plan = tnlm.BatchPlan([g], [pb.y], [f], [p])
    graph = _time_ms(lambda: plan.run(c1.n_outer), stream, reps=5)
    plan.close()
    g.close()
    return {"c1_workload": "plain TNLM-R FP32 4 x 32^3, 20 views x 64x48, patch 3^3, window 5^3, 5 iterations",
            "c1_ms_per_iteration": round(plain / c1.n_outer, 4),
            "c1_graph_ms_per_iteration": round(graph / c1.n_outer, 4)}


def batch_configs(n: int = 16, seed: int = 1005):
    """Uneven TNLM-R problems: 6-10 phases, volumes from 128x128x48 to
    256x256x96 (same 512 x 512 x 192 mm field), 20-60 views per phase (uneven
    within a problem), 384x288 or 512x384 detectors of the same 399 x 300 mm
    area; patch 3^3, window 7^3."""
    from paper_1201_2450_gb300 import synth
    rng = np.random.default_rng(seed)
    cfgs = []
    for b in range(n):
        nph = int(rng.integers(6, 11))
        k = int(rng.integers(0, 5))  # 0..4 -> 128..256 in steps of 32
        nx, nz = 128 + 32 * k, 48 + 12 * k
        nu, nv = (384, 288) if rng.uniform() < 0.5 else (512, 384)
        views = [int(v) for v in rng.integers(20, 61, size=nph)]
        cfgs.append(synth.ReconConfig(f"batch problem {b}", nph, (nx, nx, nz), 512.0 / nx, views, (nu, nv),
                                      399.4 / nu, 5e4, 1, 3, 0.02, 1.0, 3, "thorax", 2000 + b))
    return cfgs


def measure_batch(tnlm, synth, stream, n_outer: int = 20) -> dict:
    """16 uneven problems: sequential tnlm_reconstruct calls against one
    captured plan replayed n_outer times, in FP32 and in BF16 storage, with
    launch shapes tuned per problem first; BF16 error = max over problems of
    rel-L2 against the FP32 result (the FP32 path is within 1e-5 of the FP64
    oracle in the parity tests)."""
    cfgs = batch_configs()
    probs = [synth.recon_problem(c, device="cuda") for c in cfgs]
    geoms = [tnlm.Geometry(pb.geom) for pb in probs]
    ys = [pb.y.contiguous() for pb in probs]
    taus = []
    for k, g in enumerate(geoms):  # tau = 1/L per problem (20 power iterations from a seeded start)
        x0 = torch.from_numpy(synth.uniform(g.vol_shape, 3000 + k)).cuda()
        taus.append(1.0 / tnlm.tnlm_operator_norm(g, x0, 20))
        del x0
    params = [tnlm.Params(d=c.d, M=c.M, h=c.h, mu=c.mu, tau=t, n_outer=n_outer) for c, t in zip(cfgs, taus)]
    for g, p in zip(geoms, params):
        tnlm.tnlm_autotune(g, p)
    fs = [torch.zeros(g.vol_shape, device="cuda") for g in geoms]

    def seq():
        for g, y, f, p in zip(geoms, ys, fs, params):
            f.zero_()
            tnlm.tnlm_reconstruct(g, y, f, p)

    seq_ms = _time_ms(seq, stream, reps=1)
    plan = tnlm.BatchPlan(geoms, ys, fs, params)

    def run_plan(pl, xs):
        for x in xs:
            x.zero_()
        pl.run(n_outer)

    bat_ms = _time_ms(lambda: run_plan(plan, fs), stream, reps=1)
    plan.close()
    fg = [torch.zeros_like(f) for f in fs]
    gplan = tnlm.BatchPlan(geoms, ys, fg, params, grouped=True)
    grp_ms = _time_ms(lambda: run_plan(gplan, fg), stream, reps=1)
    gplan.close()
    grouped_equal = all(bool(torch.equal(a, b)) for a, b in zip(fg, fs))
    del fg
    ys16 = [y.bfloat16() for y in ys]
    fs16 = [torch.zeros(g.vol_shape, device="cuda", dtype=torch.bfloat16) for g in geoms]
    plan16 = tnlm.BatchPlan(geoms, ys16, fs16, params)
    b16_ms = _time_ms(lambda: run_plan(plan16, fs16), stream, reps=1)
    plan16.close()
    err16 = max(float(torch.linalg.vector_norm((a.float() - b).double()) / torch.linalg.vector_norm(b.double()))
                for a, b in zip(fs16, fs))
    n_it = n_outer * len(cfgs)
    voxels = sum(c.n_phases * c.vol[0] * c.vol[1] * c.vol[2] for c in cfgs)
    res = {"batch16_workload": "16 uneven TNLM-R problems (6-10 phases, 128^2x48..256^2x96, 20-60 views/phase, "
                               f"384x288 or 512x384), {n_outer} FBS iterations each, autotuned launch shapes",
           "batch16_total_voxels": voxels,
           "batch16_graph_ms": round(bat_ms, 2), "batch16_sequential_ms": round(seq_ms, 2),
           "batch16_grouped_persistent_sweep_ms": round(grp_ms, 2),
           "batch16_grouped_equals_graph_bitwise": grouped_equal,
           "batch16_graph_problem_iterations_per_s": round(n_it / (bat_ms / 1e3), 3),
           "batch16_sequential_problem_iterations_per_s": round(n_it / (seq_ms / 1e3), 3),
           "batch16_bf16_graph_ms": round(b16_ms, 2),
           "batch16_bf16_graph_problem_iterations_per_s": round(n_it / (b16_ms / 1e3), 3),
           "batch16_bf16_max_rel_l2_vs_fp32": float(f"{err16:.3e}")}
    for g in geoms:
        g.close()
    del probs, ys, fs, ys16, fs16
    torch.cuda.empty_cache()
    return res


# ---------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline and reference arm)
# ---------------------------------------------------------------------------

def cpu_baseline_sample(cfg, pb=None) -> dict:
    """Time the FP64 oracle as it stands on a bounded sample of one FBS
    iteration of the workload and extrapolate to iterations/s:
    projection and transpose of 12 views (x 360 views), one sweep on a
    3-phase 256 x 256 x 12 slab (x voxel-updates of 10 x 256^2 x 64)."""
    import oracle
    from paper_1201_2450_gb300 import synth

    oracle.build()
    geom = cfg.geometry() if pb is None else pb.geom
    truth = (pb.truth.cpu() if pb is not None else synth.rasterize(geom, synth._objects(cfg))).numpy()
    nview, nsl = 12, 12
    sub = dict(geom)
    sub["nviews"] = np.array([nview], np.int32)
    sub["angles"] = np.asarray(geom["angles"][:nview])
    G1 = oracle.Geometry(sub)
    vol1 = truth[:1].astype(np.float64)
    t0 = time.perf_counter()
    p = oracle.project(G1, vol1)
    t1 = time.perf_counter()
    oracle.backproject(G1, p)
    t2 = time.perf_counter()
    slab = truth[:3, 26:26 + nsl].astype(np.float64)
    oracle.gj_sweep(slab, slab, slab, cfg.d, cfg.M, cfg.h, cfg.mu, 1)
    t3 = time.perf_counter()
    n_views = int(np.sum(geom["nviews"]))
    per_iter = (t1 - t0) / nview * n_views + (t2 - t1) / nview * n_views + \
        (t3 - t2) * (cfg.n_phases * cfg.vol[2]) / (3 * nsl)
    return {"value": round(1.0 / per_iter, 6), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"FP64 oracle: P and P^T of {nview} views (x{n_views / nview:.0f}), one sweep on 3 phases x "
                      f"256x256x{nsl} (x{cfg.n_phases * cfg.vol[2] / (3 * nsl):.1f}); {t3 - t0:.1f} s measured, "
                      f"{per_iter:.1f} s per iteration extrapolated"}


def run_reference(args, rank, world):
    from paper_1201_2450_gb300 import synth
    if rank != 0:
        return None
    cfg = synth.C2
    for _ in range(args.warmup):
        cpu_baseline_sample(cfg)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline_sample(cfg))
    wall = time.perf_counter() - t0
    value = statistics.median(v["value"] for v in vals)
    cb = dict(vals[-1])
    cb["value"] = value
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 / value, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "reference": "FP64 CPU oracle (bounded sample, extrapolated)"},
            "cpu_baseline": cb, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0},
            "wall_s": round(wall, 1)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--phases", type=int, default=10, help="phases of the workload (10; fewer for profiling)")
    ap.add_argument("--power-iters", type=int, default=20, help="power iterations that size the step tau")
    ap.add_argument("--no-variants", action="store_true", help="skip the FDK / CGLS / TNLM-E measurements")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--storage", choices=["fp32", "bf16", "fp16"], default="fp32",
                    help="storage of the images and projections in the timed loop (arithmetic stays FP32)")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    line = run_ours(args, rank, world, local)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
