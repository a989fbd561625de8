#!/usr/bin/env python
"""Throughput of the IFGF-accelerated CFIE apply on one GB300 (one JSON line).

Workload: unit sphere 16 wavelengths across (k = 16 pi), equiangular cube-sphere
grid 6 x 256 x 256 with 8 x 8 Fejer sub-patches (N = 393,216), automatic octree
depth (~64 points per leaf, D = 6), combined-field kernel with eta = k, seeded
complex density.  The headline value is the mixed-precision apply at the
interpolation orders that reach a relative l2 error <= 1e-4 against the direct
sum (measured in the same run on sampled rows); the FP64 apply, the paper's
orders (3, 5, 5) and an end-to-end host-buffer apply are reported beside it.

A step is one operator apply y = A sigma (all stages).  Device time per step is
taken with CUDA events on the launch stream; a 256 MB buffer is written between
timed steps to flush the 129 MB L2.  With torchrun (N > 1) every rank runs an
independent replica (the apply does not shard across GPUs); value = points of
all ranks / max-over-ranks time.

Beside the headline: a four-right-hand-side apply (per-rhs throughput), the
adjoint and the vector-Jacobian product, an end-to-end apply through pinned host
buffers, off-surface evaluation, the FP64 apply, the paper's orders (3, 5, 5),
the 24-scatterer batch as one CUDA graph at the headline orders, the adaptive
octree against the uniform one on a two-density point set, and the FP64 CPU
oracle applied to the whole workload on the host cores (cpu_baseline).

--quick skips the FP64, paper-orders, CPU-oracle and adaptive-octree legs; --adaptive brings the last back.

--impl reference times the FP64 CPU oracle (the IFGF apply of Section 3.4, OpenMP
on the host cores) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CFIE matvec Mpts/s at rel err≤1e-4: mixed vs FP64 IFGF; adjoint/forward ratio"
UNIT = "Mpts/s"
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256, help="points per cube-face side")
    ap.add_argument("--wavelengths", type=float, default=16.0)
    ap.add_argument("--orders", default="5x8", help="Ps x Pang of the headline apply")
    ap.add_argument("--nc0", type=int, default=2, help="coarsest angular cone count n_C0")
    ap.add_argument("--ns0", type=int, default=1, help="coarsest radial cone count n_S0")
    ap.add_argument("--factor-mode", type=int, default=1,
                    help="0 hybrid (split factors below lambda/2), 1 combined factor on every level (the setting "
                         "of the paper's experiments), 2 split everywhere")
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--tc-fill", type=float, default=None, help="tensor-core propagation fill threshold")
    ap.add_argument("--tc-engine", type=int, default=None, help="tensor-core propagation engine: 1 tcgen05, 0 mma.sync")
    ap.add_argument("--rows", type=int, default=2000, help="direct-sum rows for the error check")
    ap.add_argument("--quick", action="store_true", help="skip the CPU legs and the FP64 timing")
    ap.add_argument("--no-batch", action="store_true", help="skip the 24-scatterer graph apply")
    ap.add_argument("--adaptive", action="store_true",
                    help="with --quick: run the adaptive-octree leg too (without its direct-sum error rows)")
    ap.add_argument("--batch-orders", default="5x8", help="Ps x Pang of the 24-scatterer graph apply")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default kernel choices instead of autotuning them on this workload")
    return ap.parse_args()


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def random_density_like(sig, seed):
    from workloads import random_density

    return random_density(sig.shape[1], sig.shape[0], seed)


def workload(args):
    from workloads import random_density, sphere_workload

    s, k = sphere_workload(args.n, 8, args.wavelengths)
    sig = random_density(s.N, args.nrhs, 2)
    return s, k, sig


def cap_sample(s, frac=8):
    """Points of the spherical cap holding 1/frac of the sphere's area (z > 1 - 2/frac)."""
    return np.nonzero(s.points[:, 2] > 1.0 - 2.0 / frac)[0]


def full_octree(s):
    """Root box (AABB midpoint, max extent * (1 + 2^-30)) and level count of the whole surface."""
    import oracle

    lo, hi = s.points.min(0), s.points.max(0)
    return {"root_center": tuple(0.5 * (lo + hi)), "root_side": float((hi - lo).max() * (1 + 2.0 ** -30)),
            "D": oracle.auto_levels(s.points)}


def oracle_cap_apply(s, k, sig, tree, Ps, Pang):
    """One oracle IFGF apply on the cap sample, on the full sphere's octree (same root box, D)."""
    import oracle

    idx = cap_sample(s)
    p = oracle.IFGFParams(k=k, Ps=Ps, Pang=Pang, nC0=tree.get("nC0", 2), nS0=tree.get("nS0", 1), levels=tree["D"],
                          identity_coef=0.5, factor_mode=tree.get("factor_mode", 0),
                          root_center=tree["root_center"], root_side=tree["root_side"])
    t = time.perf_counter()
    oracle.ifgf(s.points[idx], s.normals[idx], s.weights[idx], p, sig[:, idx])
    return len(idx), time.perf_counter() - t


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"ifgf_bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.dev), "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sm, mx, reasons = [], None, set()
        for line in open(self.path):
            c = [x.strip() for x in line.split(",")]
            if len(c) < 9:
                continue
            try:
                sm.append(float(c[1]))
                mx = float(c[2])
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), c[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


KERNEL_OF_STAGE = {"leaf": "k_leaf32p", "near": "k_near32", "cousin": "k_cousin_cs", "cousin_sum": "k_cousin_sum",
                   "prop": "k_prop_w", "prop_tc": "k_prop_t5", "prop_cs": "k_prop_cs"}
TRAFFIC_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles",
                            "dram_traffic_sphere16lambda_5x8.txt")


def tf32_peak_tflops():
    """Dense TF32 tensor peak: the measured sustained bf16 GEMM rate times the nominal TF32/bf16
    ratio (1.1 / 2.25 PFLOP/s); fallback 1.7 PFLOP/s sustained bf16."""
    bf16 = 1700.0
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            bf16 = float(json.load(f).get("bf16_tflops_sustained", bf16))
    except (OSError, ValueError):
        pass
    return bf16 * 1.1 / 2.25


def kernel_source_digest():
    """sha256 of the sources of the forward apply (its kernels, their instantiations and its host
    launch code); recorded next to ncu traffic so that stale counters are not used."""
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2112_06316_gb300", "csrc")
    h = hashlib.sha256()
    for fn in sorted(os.listdir(src)):
        if fn in ("fwd_kernels.cuh", "kernels.cuh", "apply.cu", "ifgf_internal.h") or fn.startswith("inst_"):
            with open(os.path.join(src, fn), "rb") as f:
                h.update(fn.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def recorded_traffic(stage, launches, Ps, Pang, N, args):
    """DRAM bytes (read + write) per launch of the stage's kernel from the committed ncu summary,
    only when it was taken on this workload and on the current kernel sources; else None."""
    if (Ps, Pang, N, args.nrhs, args.factor_mode, args.nc0, args.ns0) != (5, 8, 393216, 1, 1, 2, 1):
        return None
    try:
        with open(TRAFFIC_FILE) as f:
            lines = [ln.split() for ln in f if ln.strip() and not ln.startswith("#") or ln.startswith("# digest")]
    except OSError:
        return None
    digest = next((ln[2] for ln in lines if ln[:2] == ["#", "digest"]), None)
    if digest != kernel_source_digest():
        return None
    rows = [ln for ln in lines if ln and ln[0] == stage]
    if not rows:
        return None
    return float(rows[0][1])


def algorithmic_flops(info, P, nrhs, split_levels):
    """FP32-class operations the method must perform per stage (see the design notes):
    kernel evaluation 40 flops + 8 per rhs and factor; interpolation 4 P per rhs and
    factor + 100 (geometry, basis, centred factor)."""
    D = info["D"]
    nf = lambda d: 2 if split_levels[d] else 1
    leaf = info["leaf_evals"] * (40 + 8 * nrhs * nf(D))
    near = (info["near_pairs"] - info["N"]) * (40 + 8 * nrhs)
    cousin = {d: info["cousin_evals"][d] * (100 + 4 * P * nrhs * nf(d)) for d in range(3, D + 1)}
    prop = {d: info["prop_evals"][d] * (100 + 4 * P * nrhs * nf(d + 1)) for d in range(3, D)}
    return leaf, near, cousin, prop


def launches_of(stages, nrhs=1, near_blocks=0):
    """Kernel launches of one profiled mixed apply: one per stage entry, eight (one per child octant)
    for a tensor-core or cone-stationary propagation level, two for the level-D leaf stage with one
    right-hand side (the density pairs are packed first; an adaptive tree's coarser leaves take one
    each), two for the near field of an adaptive tree with block chunks (near_blocks > 0)."""
    D = max((lev for kind, lev, _ in stages if kind == "leaf"), default=0)
    return sum(8 if kind in ("prop_tc", "prop_cs") else 2 if kind == "leaf" and nrhs == 1 and lev == D
               else 2 if kind == "near" and near_blocks > 0 else 1
               for kind, lev, _ in stages)


def reduce_over_ranks(ms: float, points: float, world: int, device="cpu"):
    """Whole-job figures of independent replicas: (max over ranks of the time per step, sum over
    ranks of the points per step).  Every rank must call it (collectives of the default group)."""
    if world <= 1:
        return ms, float(points)
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    p = torch.tensor([float(points)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t.item()), float(p.item())


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    import oracle

    s, k, sig = workload(args)
    Ps, Pang = (int(v) for v in args.orders.split("x"))
    oracle.build()
    info = full_octree(s)
    info.update(nC0=args.nc0, nS0=args.ns0, factor_mode=args.factor_mode)
    n = 0
    for _ in range(args.warmup):
        oracle_cap_apply(s, k, sig, info, Ps, Pang)
    ts = []
    for _ in range(args.steps):
        n, t = oracle_cap_apply(s, k, sig, info, Ps, Pang)
        ts.append(t)
    ms = 1e3 * float(np.mean(ts))
    value = n * args.nrhs / (ms * 1e3)
    sample = (f"oracle IFGF (FP64, OpenMP) on the {n}-point spherical cap z > 0.75 of the workload, "
              f"on the full sphere's octree (D={info['D']}, same root box), orders ({Ps},{Pang},{Pang}), "
              f"nC0={args.nc0}, nS0={args.ns0}, factor mode {args.factor_mode}")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"sphere {args.wavelengths:g} wavelengths, cube-sphere 6x{args.n}x{args.n} "
                               f"(N={s.N}), orders ({Ps},{Pang},{Pang}), nC0={args.nc0}, nS0={args.ns0}, "
                               f"factor mode {args.factor_mode}, nrhs={args.nrhs}"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def adaptive_leg(args, timed, dev, Ps, Pang, rank, out):
    """The adaptive octree (leaf_max = 64, depth up to 8) against the uniform tree (the automatic depth
    and the best fixed depth) on a non-uniform point set: the unit sphere 8 wavelengths across (6 x 128
    x 128 points) and a sphere of radius 0.1 centred at (1.6, 0, 0) with as many points (a point
    density 100x higher), mixed apply at the headline orders, one right-hand side; errors against the
    direct sum on sampled rows (rank 0)."""
    import torch

    from paper_2112_06316_gb300 import Params, Plan
    from workloads import random_density, two_spheres

    s2 = two_spheres(128, 128, 0.1, 1.6)
    k2 = 8 * math.pi
    sig_np = random_density(s2.N, 1, 11)
    sig2 = torch.from_numpy(sig_np.astype(np.complex64)).to(dev)
    y2 = torch.empty_like(sig2)
    kk = max(5, args.steps // 4)
    res = {"workload": f"two spheres: unit sphere 8 wavelengths across (k={k2:.4f}), cube-sphere 6x128x128, and "
                       f"radius 0.1 at (1.6, 0, 0), 6x128x128 (density 100x); N={s2.N}; orders ({Ps},{Pang},{Pang}), "
                       f"factor mode {args.factor_mode}, one right-hand side, mixed",
           "N": s2.N, "steps": kk}
    ys = {}
    for name, kw in (("adaptive_leaf64_D8", dict(levels=8, leaf_max=64)), ("uniform_auto_depth", {}),
                     ("uniform_D7", dict(levels=7))):
        t0 = time.perf_counter()
        pl = Plan(s2.points, s2.normals, s2.weights, Params(k=k2, Ps=Ps, Pang=Pang, factor_mode=args.factor_mode, **kw))
        tb = time.perf_counter() - t0
        info = pl.info()
        t = float(np.mean(timed(lambda: pl.apply(sig2, out=y2), kk, 2)))
        pl.set_profiling(True)
        pl.apply(sig2, out=y2)
        st = pl.stage_times()
        pl.set_profiling(False)
        torch.cuda.synchronize()
        out["gpu_launches"] += launches_of(st, 1, info["near_block_chunks"]) * (kk + 2 + 1)
        assert pl.missed_lookups() == 0
        ys[name] = y2.cpu().numpy().copy()
        res[name] = {"ms_per_step": t, "value": s2.N / (t * 1e3), "D": info["D"], "plan_build_s": round(tb, 2),
                     "relevant_cones": int(sum(info["nrc"])), "near_pairs": int(info["near_pairs"]),
                     "near_block_chunks": int(info["near_block_chunks"])}
        pl.close()
    res["speedup_vs_uniform_auto"] = res["uniform_auto_depth"]["ms_per_step"] / res["adaptive_leaf64_D8"]["ms_per_step"]
    res["speedup_vs_uniform_D7"] = res["uniform_D7"]["ms_per_step"] / res["adaptive_leaf64_D8"]["ms_per_step"]
    if rank == 0 and not args.quick:
        import oracle

        oracle.build()
        rows = np.random.default_rng(12).choice(s2.N, min(args.rows, s2.N), replace=False)
        yd = oracle.direct(s2.points, s2.normals, s2.weights, k2, k2, sig_np, cI=0.5, rows=rows)
        for name, y in ys.items():
            res[name]["rel_err_vs_direct"] = float(np.linalg.norm(y.reshape(1, -1)[:, rows] - yd) / np.linalg.norm(yd))
        res["rows"] = int(len(rows))
    return res


def run_ours(args):
    import torch

    from paper_2112_06316_gb300 import Params, Plan

    rank, world, local = env_rank()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    s, k, sig = workload(args)
    N, nrhs = s.N, args.nrhs
    Ps, Pang = (int(v) for v in args.orders.split("x"))
    t0 = time.perf_counter()
    plan = Plan(s.points, s.normals, s.weights,
                Params(k=k, Ps=Ps, Pang=Pang, nC0=args.nc0, nS0=args.ns0, factor_mode=args.factor_mode))
    plan_s = time.perf_counter() - t0
    if args.tc_fill is not None:
        plan.set_tc_fill(args.tc_fill)
    if args.tc_engine is not None:
        plan.set_tc_engine(args.tc_engine)
    info = plan.info()
    P = Ps * Pang * Pang
    sig32 = torch.from_numpy(sig.astype(np.complex64)).to(dev)
    sig64 = torch.from_numpy(sig).to(dev)
    y32 = torch.empty_like(sig32)
    y64 = torch.empty_like(sig64)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        barrier()
        return [a.elapsed_time(b) for a, b in ev]

    # ---- kernel choices of the mixed apply (tensor-core fill threshold and engine, interpolation engine):
    # autotuned on this workload, outside the timed region, unless given on the command line ----
    autotune = None
    if args.tc_fill is None and args.tc_engine is None and not args.no_tune:
        from paper_2112_06316_gb300.autotune import Autotuner, tune_plan

        cache = os.path.join(tempfile.gettempdir(), f"ifgf_bench_tune_{os.getpid()}.json")
        tr = tune_plan(plan, sig32, Autotuner(cache), reps=3, force=True)
        autotune = {"config": tr.config, "ms": tr.ms, "candidates": len(tr.table),
                    "table": [[c, round(t, 4)] for c, t in tr.table]}

    # ---- headline: mixed apply ----
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    t_mixed = timed(lambda: plan.apply(sig32, out=y32), args.steps, args.warmup)
    clk = clocks.stop()
    ms, points = reduce_over_ranks(float(np.mean(t_mixed)), N * nrhs, world, dev)
    value = points / (ms * 1e3)

    # ---- several right-hand sides per apply: per-rhs throughput ----
    sig4 = torch.from_numpy(random_density_like(np.zeros((4, N)), 11).astype(np.complex64)).to(dev)
    y4 = torch.empty_like(sig4)
    t4 = timed(lambda: plan.apply(sig4, out=y4), max(3, args.steps // 5), 2)
    ms4 = float(np.mean(t4))
    multi_rhs = {"nrhs": 4, "ms_per_step": ms4, "value_per_rhs": N * 4 / (ms4 * 1e3), "unit": UNIT,
                 "speedup_per_rhs_vs_nrhs1": (N * 4 / ms4) / (N * nrhs / float(np.mean(t_mixed)))}

    # ---- per-launch device times (profiled apply) ----
    plan.set_profiling(True)
    plan.apply(sig32, out=y32)
    stages = plan.stage_times()
    plan.set_profiling(False)
    launches_per_apply = launches_of(stages)
    split = info["split"]
    leaf_f, near_f, cousin_f, prop_f = algorithmic_flops(info, P, nrhs, split)
    by_kind = {}
    for kind, lvl, t in stages:
        by_kind[kind] = by_kind.get(kind, 0.0) + t
    flops_of = {"leaf": leaf_f, "near": near_f, "cousin": sum(cousin_f.values())}
    for kind in ("prop", "prop_tc", "prop_cs"):  # CUDA-core, tensor-core, cone-stationary propagation levels
        lv = [lvl for k2, lvl, _ in stages if k2 == kind]
        if lv:
            flops_of[kind] = sum(prop_f[lvl] for lvl in lv)
    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    dom = max((kk for kk in by_kind if kk in flops_of), key=lambda kk: by_kind[kk])
    # kernel launches: both propagation kinds record one entry per level for their 8 octant launches
    n_dom = sum(8 if kind in ("prop_tc", "prop_cs") else 1 for kind, _, _ in stages if kind == dom)
    dom_ms = by_kind[dom]
    achieved = flops_of[dom] / (dom_ms * 1e-3) / 1e12
    sm_mhz = clk["sm_max_mhz"] or 2070.0
    if dom == "prop_tc":
        bound, peak, basis = "tensor", tf32_peak_tflops(), "TF32 tensor: measured sustained bf16 x 1.1/2.25"
    else:
        bound = "alu"
        peak = num_sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
        basis = (f"FP32 FMA: {num_sms} SMs (multi_processor_count of the device) x {FP32_LANES_PER_SM} lanes "
                 f"x 2 flops x {sm_mhz:g} MHz (maximum SM clock)")
    roofline = {"bound": bound, "kernel": KERNEL_OF_STAGE.get(dom, dom), "stage": dom,
                "launches_per_apply": n_dom, "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": recorded_traffic(dom, n_dom, Ps, Pang, N, args),
                "peak_basis": basis,
                "all_stages_ms": {kk: round(v, 4) for kk, v in by_kind.items()},
                "per_launch_ms": [[kk, lvl, round(t, 4)] for kk, lvl, t in stages],
                "all_stages_tflops": {kk: round(flops_of[kk] / (by_kind[kk] * 1e-3) / 1e12, 3)
                                      for kk in flops_of if kk in by_kind}}

    # ---- adjoint (mixed) and vector-Jacobian product on the same plan ----
    g32 = torch.from_numpy(random_density_like(sig, 7).astype(np.complex64)).to(dev)
    a32 = torch.empty_like(g32)
    plan.adjoint(g32, out=a32)  # builds the anterpolation lists once (host)
    t_adj = timed(lambda: plan.adjoint(g32, out=a32), max(3, args.steps // 4), 2)
    adj_ms = float(np.mean(t_adj))
    plan.set_profiling(True)
    plan.adjoint(g32, out=a32)
    adj_stages = plan.stage_times()
    plan.set_profiling(False)
    # the autograd backward: gradient in sigma and k from the forward state saved by the forward apply
    _, state = plan.apply_with_state(sig32)
    t_vjp = timed(lambda: plan.vjp_from_state(state, g32), max(3, args.steps // 4), 1)
    # ifgf_apply_vjp, which re-runs the forward apply first (callers without a saved state)
    t_vjp_full = timed(lambda: plan.vjp(sig32, g32), 3, 1)
    del state
    adjoint = {"ms_per_step": adj_ms, "adjoint_forward_ratio": adj_ms / ms,
               "vjp_ms_per_step": float(np.mean(t_vjp)), "vjp_forward_ratio": float(np.mean(t_vjp)) / ms,
               "vjp_note": "backward of the autograd function: A^H g and Re <g, dA/dk sigma> from the saved forward "
                           "state (ifgf_apply_vjp_ws)",
               "vjp_with_forward_ms_per_step": float(np.mean(t_vjp_full)),
               "stages_ms": {kk: round(sum(t for k2, _, t in adj_stages if k2 == kk), 4)
                             for kk in {k2 for k2, _, _ in adj_stages}}}

    # ---- end to end through host (pinned) buffers ----
    hs = torch.from_numpy(sig.astype(np.complex64)).pin_memory()
    hy = torch.empty_like(hs).pin_memory()
    dsig = torch.empty_like(sig32)

    def e2e_step():
        dsig.copy_(hs, non_blocking=True)
        plan.apply(dsig, out=y32)
        hy.copy_(y32, non_blocking=True)

    t_e2e = timed(e2e_step, max(3, args.steps // 4), 2)
    e2e_ms = float(np.mean(t_e2e))
    e2e = {"value": N * nrhs * world / (e2e_ms * 1e3), "unit": UNIT, "ms_per_step": e2e_ms,
           "h2d_bytes_per_step": int(hs.numel() * hs.element_size()),
           "d2h_bytes_per_step": int(hy.numel() * hy.element_size())}

    # ---- off-surface evaluation of the same density (mixed): far field on the 200 x 200 direction
    # grid of Eq. SphereGrid, combined-layer potential on a 200 x 200 plane z = 1.5 (Eq. PlanarGrid) ----
    pol, az = np.meshgrid(np.linspace(0.0, math.pi, 200), np.linspace(0.0, 2 * math.pi, 200), indexing="ij")
    xh = torch.from_numpy(np.stack([np.sin(pol) * np.cos(az), np.sin(pol) * np.sin(az), np.cos(pol)],
                                   -1).reshape(-1, 3)).to(dev)
    gx, gy = np.meshgrid(np.linspace(-3.0, 3.0, 200), np.linspace(-3.0, 3.0, 200), indexing="ij")
    plane = torch.from_numpy(np.stack([gx.ravel(), gy.ravel(), np.full(gx.size, 1.5)], -1)).to(dev)
    ff = torch.empty((nrhs, xh.shape[0]), dtype=torch.complex64, device=dev)
    nf = torch.empty((nrhs, plane.shape[0]), dtype=torch.complex64, device=dev)
    k_off = max(3, args.steps // 10)
    t_ff = float(np.mean(timed(lambda: plan.far_field(sig32, xh, out=ff), k_off, 2)))
    t_nf = float(np.mean(timed(lambda: plan.field(sig32, plane, out=nf), k_off, 2)))
    off_surface = {
        "far_field": {"targets": int(xh.shape[0]), "ms_per_step": t_ff,
                      "Gpairs_per_s": N * nrhs * xh.shape[0] / (t_ff * 1e6)},
        "plane_potential": {"targets": int(plane.shape[0]), "ms_per_step": t_nf,
                            "Gpairs_per_s": N * nrhs * plane.shape[0] / (t_nf * 1e6)},
        "note": "direct sums over all N sources (ifgf_far_field, ifgf_field), mixed precision"}

    # ---- the same far field from the level-3 interpolants (plan option far_field=1: the is = 0 cone
    # segments of level 3 kept relevant), against the direct sum above ----
    t0 = time.perf_counter()
    plan_ff = Plan(s.points, s.normals, s.weights, Params(k=k, Ps=Ps, Pang=Pang, nC0=args.nc0, nS0=args.ns0,
                                                          factor_mode=args.factor_mode, far_field=1))
    ff_plan_s = time.perf_counter() - t0
    if args.tc_fill is not None:
        plan_ff.set_tc_fill(args.tc_fill)
    if args.tc_engine is not None:
        plan_ff.set_tc_engine(args.tc_engine)
    ffi = torch.empty_like(ff)
    t_ffi = float(np.mean(timed(lambda: plan_ff.far_field_ifgf(sig32, xh, out=ffi), k_off, 2)))
    t_app_ff = float(np.mean(timed(lambda: plan_ff.apply(sig32, out=y32), k_off, 2)))
    plan_ff.set_profiling(True)
    plan_ff.apply(sig32, out=y32)
    ff_apply_launches = launches_of(plan_ff.stage_times())
    plan_ff.far_field_ifgf(sig32, xh, out=ffi)
    up_stages = plan_ff.stage_times()
    plan_ff.set_profiling(False)
    torch.cuda.synchronize()
    d_ff = (ffi - ff).abs()
    off_surface["far_field_ifgf"] = {
        "targets": int(xh.shape[0]), "ms_per_step": t_ffi, "speedup_vs_direct_sum": t_ff / t_ffi,
        "rel_err_vs_direct_sum_l2": float(torch.linalg.vector_norm(ffi - ff) / torch.linalg.vector_norm(ff)),
        "rel_err_vs_direct_sum_max": float(d_ff.max() / ff.abs().max()),
        "upward_pass_ms": round(sum(t for _, _, t in up_stages), 4),
        "apply_ms_of_the_far_field_plan": t_app_ff, "plan_build_s": round(ff_plan_s, 2),
        "nrc_level3": {"with_far_field_cones": plan_ff.info()["nrc"][3], "without": info["nrc"][3]},
        "note": "ifgf_far_field_ifgf: upward pass (leaf expansions, propagation) plus one warp per direction "
                "over the level-3 boxes, mixed precision"}
    assert plan_ff.missed_lookups() == 0
    # ---- the plane potential with the plane's points inside the octree (zero-weight targets) ----
    t0 = time.perf_counter()
    plan_nf = Plan.with_targets(s.points, s.normals, s.weights, plane.cpu().numpy(),
                                Params(k=k, Ps=Ps, Pang=Pang, nC0=args.nc0, nS0=args.ns0,
                                       factor_mode=args.factor_mode))
    nf_plan_s = time.perf_counter() - t0
    if args.tc_fill is not None:
        plan_nf.set_tc_fill(args.tc_fill)
    if args.tc_engine is not None:
        plan_nf.set_tc_engine(args.tc_engine)
    nfi = torch.empty_like(nf)
    t_nfi = float(np.mean(timed(lambda: plan_nf.field_ifgf(sig32, out=nfi), k_off, 2)))
    plan_nf.set_profiling(True)
    plan_nf.field_ifgf(sig32, out=nfi)
    nf_launches = launches_of(plan_nf.stage_times())
    plan_nf.set_profiling(False)
    torch.cuda.synchronize()
    off_surface["plane_potential_ifgf"] = {
        "targets": int(plane.shape[0]), "ms_per_step": t_nfi, "speedup_vs_direct_sum": t_nf / t_nfi,
        "rel_err_vs_direct_sum_l2": float(torch.linalg.vector_norm(nfi - nf) / torch.linalg.vector_norm(nf)),
        "rel_err_vs_direct_sum_max": float((nfi - nf).abs().max() / nf.abs().max()),
        "plan_build_s": round(nf_plan_s, 2), "D": plan_nf.info()["D"],
        "note": "ifgf_field_ifgf: the plane's points join the octree with weight 0; one apply over sources "
                "and targets, mixed precision"}
    assert plan_nf.missed_lookups() == 0
    plan_nf.close()
    k_ffi = k_off + 2 + 1  # timed calls and warm-up, and the profiled call
    ff_launches = launches_of(up_stages) + 1  # the upward pass and k_far_ifgf
    plan_ff.close()

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"sphere {args.wavelengths:g} wavelengths across (k={k:.4f}), cube-sphere "
                                  f"6x{args.n}x{args.n} with 8x8 Fejer sub-patches, N={N}, D={info['D']}, "
                                  f"orders ({Ps},{Pang},{Pang}), nC0={args.nc0}, nS0={args.ns0}, "
                                  f"factor mode {args.factor_mode} (1: combined factor on every level), eta=k, "
                                  f"nrhs={nrhs}",
                      "kernel_choices": autotune["config"] if autotune else
                      {"tc_fill": 0.4 if args.tc_fill is None else args.tc_fill,
                       "tc_engine": 1 if args.tc_engine is None else args.tc_engine, "interp_engine": 1},
                      "l2_flush_between_steps": True, "parallelism": "replicas" if world > 1 else "single",
                      "plan_build_s": round(plan_s, 2)},
           "roofline": roofline, "e2e": e2e, "multi_rhs": multi_rhs, "adjoint": adjoint, "off_surface": off_surface,
           "autotune": autotune,
           "adjoint_forward_ratio": adjoint["adjoint_forward_ratio"],
           # gather, sum and (when the sources are split into chunks) the reduction per off-surface call
           "gpu_launches": launches_per_apply * (args.steps + len(t4)) + len(adj_stages) * max(3, args.steps // 4)
                           + 2 * 3 * k_off + ff_launches * k_ffi + ff_apply_launches * (k_off + 3)
                           + nf_launches * (k_off + 3),
           "clocks": clk}

    if not args.quick:
        # ---- FP64 apply (same plan) ----
        k64 = max(3, args.steps // 20)
        t64 = timed(lambda: plan.apply(sig64, out=y64), k64, 1)
        ms64 = float(np.mean(t64))
        out["fp64"] = {"value": N * nrhs * world / (ms64 * 1e3), "ms_per_step": ms64, "steps": k64}
        out["mixed_vs_fp64_speedup"] = ms64 / ms
        out["gpu_launches"] += launches_per_apply * k64
        # ---- paper orders (3,5,5) for context ----
        plan35 = Plan(s.points, s.normals, s.weights, Params(k=k, factor_mode=args.factor_mode))
        y35 = torch.empty_like(sig32)
        t35 = timed(lambda: plan35.apply(sig32, out=y35), max(5, args.steps // 4), 2)
        out["paper_orders_3x5"] = {"value": N * nrhs * world / (float(np.mean(t35)) * 1e3),
                                   "ms_per_step": float(np.mean(t35))}
        out["gpu_launches"] += len(stages) * max(5, args.steps // 4)
        assert plan.missed_lookups() == 0 and plan35.missed_lookups() == 0
        torch.cuda.synchronize()
        if rank == 0:
            # ---- CPU legs (oracle): direct-sum rows for the error check, IFGF baseline ----
            import oracle

            oracle.build()
            rows = np.random.default_rng(0).choice(N, min(args.rows, N), replace=False)
            t = time.perf_counter()
            yd = oracle.direct(s.points, s.normals, s.weights, k, k, sig, cI=0.5, rows=rows)
            t_direct = time.perf_counter() - t

            def err(y):
                return float(np.linalg.norm(y.cpu().numpy()[:, rows] - yd) / np.linalg.norm(yd))

            out["rel_err_vs_direct"] = {"mixed": err(y32), "fp64": err(y64), "paper_orders_3x5_mixed": err(y35),
                                        "rows": int(len(rows))}
            out["fp64"]["rel_err_vs_direct"] = out["rel_err_vs_direct"]["fp64"]
            out["paper_orders_3x5"]["rel_err_vs_direct"] = out["rel_err_vs_direct"]["paper_orders_3x5_mixed"]
            # the oracle IFGF on the whole workload (same orders, cone grid and factor mode), timed once
            # (about 10-20 s on the host cores); a second apply when the first took under 15 s
            po = oracle.IFGFParams(k=k, Ps=Ps, Pang=Pang, nC0=args.nc0, nS0=args.ns0, factor_mode=args.factor_mode,
                                   identity_coef=0.5)
            t_or = []
            while True:
                t = time.perf_counter()
                y_or, _ = oracle.ifgf(s.points, s.normals, s.weights, po, sig)
                t_or.append(time.perf_counter() - t)
                if len(t_or) >= 2 or t_or[0] >= 15.0:
                    break
            t_cpu = float(np.mean(t_or))
            e_or = y32.cpu().numpy() - y_or
            out["rel_err_vs_oracle"] = {"mixed_l2": float(np.linalg.norm(e_or) / np.linalg.norm(y_or)),
                                        "mixed_max": float(np.abs(e_or).max() / np.abs(y_or).max())}
            out["cpu_baseline"] = {
                "value": N * nrhs / (t_cpu * 1e6), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                "sample": f"the whole workload: {len(t_or)} oracle IFGF apply(s) (FP64, OpenMP) of all N={N} points, "
                          f"orders ({Ps},{Pang},{Pang}), factor mode {args.factor_mode}; {t_cpu:.1f} s each",
                "direct_sum_rows_per_s": len(rows) / t_direct}
        plan35.close()
    if not args.quick or args.adaptive:
        out["adaptive_octree"] = adaptive_leg(args, timed, dev, Ps, Pang, rank, out)
    # ---- the corrected operator: rectangular-polar correction built on the GPU, applied by K5 in
    # every apply (the operator GMRES uses in the sound-soft solve) ----
    from paper_2112_06316_gb300 import rp_correction
    from workloads import patch_node_index

    t0 = time.perf_counter()
    rpc = rp_correction(s.points, s.normals, s.weights, patch_node_index(s), 8, k, k,
                        delta=math.pi / (2 * (args.n // 8)), device=True)
    rp_s = time.perf_counter() - t0
    nnz = int(rpc[0][-1])
    t0 = time.perf_counter()
    plan.set_correction(*rpc)
    attach_s = time.perf_counter() - t0
    del rpc
    t_corr = timed(lambda: plan.apply(sig32, out=y32), max(5, args.steps // 4), 2)
    plan.set_profiling(True)
    kspmv = []
    for _ in range(5):
        plan.apply(sig32, out=y32)
        kspmv += [t for kd, _, t in plan.stage_times() if kd == "correction"]
    plan.set_profiling(False)
    k5_ms = float(np.median(kspmv))
    k5_bytes = nnz * 12 + N * nrhs * 16  # complex64 value + int32 column per entry; sigma read, y updated
    hbm = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            hbm = float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        hbm = 6800.0
    out["corrected_apply"] = {
        "value": N * nrhs / (float(np.mean(t_corr)) * 1e3), "unit": UNIT, "ms_per_step": float(np.mean(t_corr)),
        "correction_nnz": nnz, "rp_precompute_gpu_s": round(rp_s, 2), "attach_s": round(attach_s, 2),
        "k_spmv": {"ms": k5_ms, "bytes_model": "nnz x 12 B + N x nrhs x 16 B", "bytes": k5_bytes,
                   "GBps": k5_bytes / (k5_ms * 1e-3) / 1e9, "peak_GBps": hbm,
                   "frac": k5_bytes / (k5_ms * 1e-3) / 1e9 / hbm}}
    out["gpu_launches"] += (launches_per_apply + 1) * (len(t_corr) + 5)
    plan.set_correction(np.zeros(N + 1, np.int64), np.zeros(0, np.int32), np.zeros(0, complex))
    if not args.no_batch:
        from paper_2112_06316_gb300 import Group
        from workloads import random_density as _rd, scatterer_batch

        bPs, bPang = (int(v) for v in args.batch_orders.split("x"))
        bodies = scatterer_batch(seed=3)
        t0 = time.perf_counter()
        bplans = [Plan(b.points, b.normals, b.weights, Params(k=kb, Ps=bPs, Pang=bPang, factor_mode=args.factor_mode))
                  for b, kb in bodies]
        bsig_h = [_rd(b.N, 4, 300 + i) for i, (b, _) in enumerate(bodies)]
        bsig = [torch.from_numpy(x.astype(np.complex64)).to(dev) for x in bsig_h]
        bout = [torch.empty_like(x) for x in bsig]
        build_s = time.perf_counter() - t0
        grp = Group(bplans)
        tb = timed(lambda: grp.apply(bsig, bout), max(3, args.steps // 10), 2)
        npts = sum(b.N for b, _ in bodies) * 4
        batch = {"value": npts / (float(np.mean(tb)) * 1e3), "unit": UNIT, "ms_per_step": float(np.mean(tb)),
                 "bodies": len(bodies), "points_x_rhs": npts, "nrhs_per_body": 4,
                 "orders": f"{bPs}x{bPang}", "plan_build_s": round(build_s, 1)}
        if rank == 0 and not args.quick:
            import oracle

            # error of every body's first right-hand side against 200 direct-sum rows
            errs = []
            for i, (b, kb) in enumerate(bodies):
                r = np.random.default_rng(10 + i).choice(b.N, min(200, b.N), replace=False)
                yd = oracle.direct(b.points, b.normals, b.weights, kb, kb, bsig_h[i][:1], cI=0.5, rows=r)
                yb = bout[i][:1].cpu().numpy()[:, r]
                errs.append(float(np.linalg.norm(yb - yd) / np.linalg.norm(yd)))
            batch["rel_err_vs_direct_max_over_bodies"] = max(errs)
            batch["rel_err_vs_direct_median"] = float(np.median(errs))
        out["batch_24_scatterers"] = batch
        nl = 0
        for bp, x in zip(bplans, bsig):  # launches of one graph replay, counted from profiled applies
            bp.set_profiling(True)
            bp.apply(x)
            nl += launches_of(bp.stage_times(), nrhs=int(x.shape[0]) if x.dim() > 1 else 1)
            bp.set_profiling(False)
        out["gpu_launches"] += nl * len(tb)
        grp.close()
        for bp in bplans:
            bp.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    plan.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
