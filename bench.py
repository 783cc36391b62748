"""Benchmark: near-field correction entries per second on one GB300.

Headline workload (one step = one full correction build, all four kernels S, D, S', D'):
the ellipsoid with semi-axes (2, 1, 0.5) on an 81,920-patch icosahedral mesh, order
p = 6 (21 nodes per patch, 1,720,320 nodes), every node a target (on-surface rows with
the principal-value jump).  Inputs are seeded and synthetic.  The timed region starts
with geometry and targets resident in device memory and ends with the four CSR matrices
(~6.5e8 entries each) resident in device memory: near list, per-patch precompute,
per-pair stage, CSR assembly.  A 512 MB write flushes L2 between timed steps, outside the
timed region (the CSR, ~23 GB, is far larger than L2 anyway).

Beside the headline: the same build in mixed precision; the end-to-end rate through the
C ABI with host buffers; the correction SpMV of this workload against HBM bandwidth; the
star surface (1280 patches, 200k off-surface targets) and the wavy torus (20,480
patches, p = 8) in FP64 and mixed; the fused apply and the density-given evaluation on
the star; the 64-surface batch; the stellarator of the paper's throughput table.

Output: one JSON line (rank 0).  `--impl reference` times the CPU oracle instead, on a
bounded sample of the headline workload.  With torchrun (N > 1) the targets of the one
problem are split into contiguous row blocks, one per rank (every rank holds the whole
geometry; no collective in the data path); the step time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "near-correction entries/s at 1e-10 rel err; mixed vs FP64 on 1 GB300"
UNIT = "entries/s"
WORKLOAD = "ellipsoid81920_p6_1.72M_onsurface_SDSpDp"
P = 6
KERNELS = ("S", "D", "SP", "DP")
SEED = 20241115
# DRAM bytes per (target, patch) pair of the FP64 per-pair kernel at p = 6, from a one-pass
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum over the launch / its pairs),
# valid only for the kernel sources whose hash is given; otherwise reported as null.
TRAFFIC_CAPTURE = {"sources_sha16": "450d4754ced8ce17", "bytes_per_pair": 1663.0,
                   "capture": "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum, k_pairs_tile<6, false, 5> "
                              "on the 5,120-patch ellipsoid (4,347,204 pairs, 3.318 GB read + 3.910 GB written), "
                              "scaled by pairs"}


def workload(levels: int = 6):
    """The ellipsoid (2, 1, 0.5) on 20 * 4^levels patches (81,920 at the default 6), every
    node a target; smaller levels give the same workload shape for profiling captures."""
    from paper_2411_08342_gb300 import workloads as W
    return W.ellipsoid81920(P, levels)


def pair_kernel_sha16() -> str:
    h = hashlib.sha256()
    for f in ("rrq_pairs_tile.cuh", "rrq_pairs.cuh", "rrq_internal.cuh", "rrq_pairs_p6.cu"):
        with open(os.path.join(ROOT, "paper_2411_08342_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def dist_env():
    r = int(os.environ.get("RANK", "0"))
    w = int(os.environ.get("WORLD_SIZE", "1"))
    lr = int(os.environ.get("LOCAL_RANK", str(r)))
    return r, w, lr


def reduce_max(v: float, world: int, device=None) -> float:
    """Maximum over ranks (identity on one rank)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(v: float, world: int, device=None) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in the background."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def flops_per_pair(p: int) -> float:
    """Algorithmic FP64 flops of one (target, patch) pair for all four kernels, counted
    from the loops of the per-pair stage (an FMA is 2 flops; work that the kernel repeats
    but need not is counted once).  Not counted: the graded Omega_0 panels and the
    upsampled rule of far edges (their cost depends on the geometry), index arithmetic."""
    np_ = p * (p + 1) // 2
    pt = 2 * p
    njk = (p + 1) * (p + 2) // 2
    ns = 3 * pt
    n1, n2 = njk - 1, njk - 3                          # harmonics (j, k >= 0) with j >= 1, j >= 2
    # Step 6: V (3 FMA x complex) for j >= 1; for j >= 2 the product (0, d)(0, h) (18 FMA),
    # Q and the w3 (nu'.d) sum of dQ/dnu' from it (8 FMA each), sum w1 h (6 FMA)
    line = ns * (12 * n1 + 80 * n2)
    # Step 7: per (l, m >= 1), sum over (j, k): 5 flops for the psi term, 67 with Q, dQ, dS (j >= 2)
    trans = 0
    for l in range(1, p + 1):
        for m in range(1, l + 1):
            for j in range(1, l + 1):
                kmin, kmax = max(-j, m - (l - j)), min(j, m + (l - j))
                trans += max(0, kmax - kmin + 1) * (67 if j >= 2 else 5)
    trans += np_ * 100                                 # I[gamma] and its nu' derivative per (l, m)
    # Step 8: per (node, (l, m)) 4-term dot products for D, D', S', S; jump and smooth rule per node
    rows = np_ * np_ * 34 + np_ * 60
    weights = 3 * (pt * pt * 4 + pt * 30)              # lambda = V^-T I for m = 1, 3 and the ratios
    moments = 3 * 20 * pt                              # J_i, K_i recurrences
    harm = ns * 12 + njk * (8 + 36)                    # samples, target table, gradients, Hessians
    u_choice = (np_ + ns) * 10
    root = 3 * 4 * (48 * p + 20)                       # ~4 Newton steps on the complex edge polynomial
    return float(line + trans + rows + weights + moments + harm + u_choice + root)


def rank_targets(tg, rank: int, world: int):
    """The contiguous row block of this rank (all targets on one rank)."""
    from paper_2411_08342_gb300 import workloads as W
    from paper_2411_08342_gb300.shard import row_block
    lo, hi = row_block(tg.n, rank, world)
    return W.Targets(tg.xyz[lo:hi], tg.nrm[lo:hi], tg.self_node[lo:hi]), (lo, hi)


def upload(ctx, d, tg, dev):
    from paper_2411_08342_gb300 import rrq
    a = rrq.device_inputs(d, tg, device=str(dev))
    surf = ctx.surface(a["order"], a["node_off"], a["xyz"], a["nrm"], a["wts"], d.ref_uv)
    targ = ctx.targets(a["txyz"], a["tnrm"], a["tself"])
    return a, surf, targ


def time_builds(ctx, surf, targ, dev, flush, steps: int, warmup: int, mixed: bool = False, kernels=KERNELS):
    """CUDA-event times (ms) of `steps` builds after `warmup` untimed ones, an L2 flush
    before each; with the per-pair stage time of each build, entries and pairs."""
    import torch
    stream = torch.cuda.current_stream(dev)
    nnz = npairs = 0
    for _ in range(warmup):
        csr = ctx.build_corrections(surf, targ, kernels, mixed=mixed)
        ctx.csr_free(csr)
    torch.cuda.synchronize(dev)
    times, pair_ms = [], []
    for _ in range(steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        csr = ctx.build_corrections(surf, targ, kernels, mixed=mixed)
        e1.record(stream)
        e1.synchronize()
        nnz, npairs = csr.nnz, csr.npairs
        ctx.csr_free(csr)
        times.append(e0.elapsed_time(e1))
        pair_ms.append(ctx.diagnostics()["ms_pairs"])
    return times, pair_ms, nnz, npairs, ctx.diagnostics()


def autotune(ctx, surf, targ, p):
    """One-time autotuning of the per-pair launch shapes (kept in the context)."""
    tuned = {}
    for m in (False, True):
        b = ctx.batch([surf], [targ], KERNELS, mixed=m, autotune=True)
        info = b.info()
        b.close()
        tuned["mixed" if m else "fp64"] = {"tile": info["tile"][p], "persistent": info["persistent"][p],
                                           "ms_autotune": info["ms_autotune"]}
    return tuned


def bench_gpu(args):
    import torch

    from paper_2411_08342_gb300 import rrq
    rank, world, lrank = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", lrank))
    torch.cuda.set_device(lrank)
    dev = torch.device("cuda", lrank)
    d, tg_all = workload(args.levels)
    tg, (lo, hi) = rank_targets(tg_all, rank, world)
    ctx = rrq.Context(lrank)
    arrs, surf, targ = upload(ctx, d, tg, dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    tuned = None if args.no_autotune else autotune(ctx, surf, targ, P)
    peak = ctx.fma_peak_tflops(fp32=False)
    peak32 = ctx.fma_peak_tflops(fp32=True)

    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(lrank)
    clocks.start()
    time.sleep(0.3)
    times, pair_ms, nnz, npairs, diag = time_builds(ctx, surf, targ, dev, flush, args.steps, args.warmup)
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    msteps = max(2, min(args.steps, 3))
    mtimes, mpair_ms, _, _, mdiag = time_builds(ctx, surf, targ, dev, flush, msteps, 1, mixed=True)
    ms_step = reduce_max(sum(times) / len(times), world, dev)
    entries = nnz * len(KERNELS)
    total_entries = reduce_sum(float(entries), world, dev)
    value = total_entries / (ms_step * 1e-3)
    ms_mixed = reduce_max(sum(mtimes) / len(mtimes), world, dev)

    # roofline of the dominant kernel: the per-pair stage (k_roots + k_uside + k_pairs_tile),
    # FP64 ALU bound; algorithmic flops per pair from the loop count model
    fpp = flops_per_pair(P)
    pair_s = sum(pair_ms) / len(pair_ms) * 1e-3
    achieved = fpp * npairs / pair_s / 1e12
    sha = pair_kernel_sha16()
    cap = TRAFFIC_CAPTURE
    traffic = cap["bytes_per_pair"] * npairs if (cap["bytes_per_pair"] and cap["sources_sha16"] == sha) else None
    launches = diag.get("kernel_launches", None)

    e2e = None
    if not args.no_e2e:
        try:
            e2e = e2e_leg(ctx, d, tg, nnz, dev, flush, args, world, total_entries)
        except (RuntimeError, MemoryError) as ex:   # e.g. page-locked host memory exhausted
            e2e = {"error": f"{type(ex).__name__}: {ex}"[:300]}
    spmv = None if args.no_apply else spmv_leg(ctx, surf, targ, d, tg, dev)
    legs = {}
    if not args.no_extra and world == 1:
        legs["star1280"] = star_leg(ctx, dev, flush, args)
        legs["torus"] = torus_leg(ctx, dev, flush, args)
    if not args.no_batched and world == 1:
        legs["batched"] = batched_leg(ctx, dev)
        legs["stellarator"] = stellarator_leg(ctx, dev)
        legs["translation"] = translation_leg(ctx, dev)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "strong" if world > 1 else "weak",
        "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded closed-form ellipsoid; every node a target)",
        "config": {"workload": WORKLOAD if args.levels == 6 else f"ellipsoid{d.npatch}_p6_onsurface_SDSpDp",
                   "patches": d.npatch, "p": P, "nodes": d.nnode, "targets": tg_all.n,
                   "rank_rows": [lo, hi], "kernels": list(KERNELS), "pairs": npairs, "nnz_per_kernel": nnz,
                   "l2": "512 MB flush between timed steps; CSR (~23 GB) larger than L2",
                   "parallelism": f"row blocks x{world}" if world > 1 else "single GPU"},
        "e2e": e2e,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": traffic,
                     "traffic_note": (f"{cap['bytes_per_pair']} DRAM bytes per pair x {npairs} pairs; {cap['capture']}"
                                      if traffic is not None else
                                      f"null: no DRAM capture of the current per-pair kernel sources ({sha})"),
                     "kernel": "k_roots<6> + k_uside<6> + k_pairs_tile<6, false, T> (one per-pair stage)",
                     "peak_note": "of measured: FP64 FMA peak of this GPU (rrq_measure_fma_peak); FP32 FMA peak "
                                  "%.1f TFLOP/s" % peak32,
                     "flops_per_pair": fpp, "kernel_ms": pair_s * 1e3},
        "stage_ms": {"precompute": diag["ms_precompute"], "near_and_items": diag["ms_near"], "pairs": diag["ms_pairs"]},
        "fit_kappa_max": diag["kappa_max"],
        "accuracy": {
            "reference": "binary128 build of the oracle (same algorithm, rounding unit 2^-113), "
                         "tests/test_gpu_parity.py::test_full_size_ellipsoid_sampled, 100 sampled rows",
            "apply_E_true": "3.5e-12 (D), 2.6e-12 (S'), 8.7e-13 (D'), 1.4e-15 (S); the FP64 oracle's own: 1.1e-12, "
                            "7.9e-13, 3.0e-13, 1.1e-15: the corrections applied to a random Y_l^m density, "
                            "relative to the sums they correct",
            "row_E_true": "1.9e-6 (D), 1.7e-6 (S'), 4.7e-8 (S), 2.0e-10 (D'); the FP64 oracle's own: 1.9e-6, 1.3e-6, "
                          "5.0e-8, 2.4e-10 (binary64 rows of this formulation lose digits on these stretched "
                          "patches, Sec. 5.1 eq. interpolationerror)",
            "gate": "E_true <= max(1e-10, 4 x the FP64 oracle's E_true), rows and applies"},
        "launch_shape": tuned,
        "clocks": clk,
        "gpu_launches": launches * args.steps if launches is not None else None,
        "points_per_s": world * tg.n / (ms_step * 1e-3) if world == 1 else tg_all.n / (ms_step * 1e-3),
        "mixed": {"value": total_entries / (ms_mixed * 1e-3), "unit": UNIT, "ms_per_step": ms_mixed,
                  "steps": msteps, "speedup_vs_fp64": ms_step / ms_mixed,
                  "stage_ms": {"precompute": mdiag["ms_precompute"], "near_and_items": mdiag["ms_near"],
                               "pairs": mdiag["ms_pairs"]},
                  "precision": "line integrals, translations and fit contraction in double-float FP32 "
                               "(about 48 bits); roots, recurrences, Omega_0, harmonics, smooth rule FP64",
                  "accuracy": "rows and applies within max(1e-10, 32 x the FP64 oracle's error against the "
                              "binary128 oracle) (tests/test_gpu_mixed.py)"},
        "spmv": spmv,
    }
    line.update(legs)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_targets)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def spmv_leg(ctx, surf, targ, d, tg, dev, reps: int = 3) -> dict:
    """The correction alone (rrq_apply_correction: out = C sigma, one warp per row) for each
    kernel on this workload's FP64 corrections, against the measured HBM copy bandwidth;
    algorithmic bytes: 8 (value) + 4 (column) per entry, the row pointers, the output, and
    sigma once.  Kernel times by the library's CUDA events."""
    import torch
    csr = ctx.build_corrections(surf, targ, KERNELS)
    nnz = csr.nnz
    sig = torch.as_tensor(np.random.default_rng(SEED + 7).standard_normal(d.nnode), dtype=torch.float64, device=dev)
    out = torch.empty(tg.n, dtype=torch.float64, device=dev)
    ms = []
    for k in KERNELS:
        for it in range(reps + 1):
            ctx.apply_correction(csr, k, sig, out)
            if it > 0:
                ms.append(ctx.diagnostics()["ms_apply_spmv"])
    ctx.csr_free(csr)
    t = statistics.median(ms)
    nbytes = nnz * 12 + (tg.n + 1) * 8 + tg.n * 8 + d.nnode * 8
    peak = measured_peaks().get("hbm_gbs")
    gbs = nbytes / (t * 1e-3) / 1e9
    return {"ms": t, "nnz": nnz, "bytes": nbytes, "achieved_gbs": gbs, "peak_gbs": peak,
            "frac": gbs / peak if peak else None,
            "peak_note": ("of measured HBM copy bandwidth (MEASURED_PEAKS.json)" if measured_peaks()["source"] == "measured"
                          else "of fallback HBM copy bandwidth (6.8 TB/s; no MEASURED_PEAKS.json on this machine)"),
            "entries_per_s": nnz / (t * 1e-3)}


def star_leg(ctx, dev, flush, args) -> dict:
    """Star surface (1280 patches, p = 6, 200,000 off-surface targets at 10^-k h): FP64 and
    mixed builds, the fused apply and the density-given evaluation."""
    from paper_2411_08342_gb300 import workloads as W
    d, tg = W.star1280(P, 200_000, seed=SEED)
    a, surf, targ = upload(ctx, d, tg, dev)
    autotune(ctx, surf, targ, P)
    t, pm, nnz, npairs, dg = time_builds(ctx, surf, targ, dev, flush, 3, 2)
    tm, _, _, _, _ = time_builds(ctx, surf, targ, dev, flush, 3, 1, mixed=True)
    ms, mm = sum(t) / len(t), sum(tm) / len(tm)
    fpp = flops_per_pair(P)
    out = {"workload": "star1280_p6_200k_offsurface_SDSpDp", "pairs": npairs, "nnz_per_kernel": nnz,
           "fp64": {"value": 4 * nnz / (ms * 1e-3), "unit": UNIT, "ms": ms,
                    "pair_stage_tflops": fpp * npairs / (sum(pm) / len(pm) * 1e-3) / 1e12},
           "mixed": {"value": 4 * nnz / (mm * 1e-3), "unit": UNIT, "ms": mm, "speedup_vs_fp64": ms / mm}}
    if not args.no_apply:
        out["apply"] = apply_leg(ctx, surf, targ, d, tg, dev)
        out["evaluate_near"] = evaluate_leg(ctx, surf, targ, d, tg, dev, ms)
    return out


def torus_leg(ctx, dev, flush, args) -> dict:
    """Wavy torus (20,480 patches, p = 8; 737,280 on-surface nodes and 200,000 off-surface
    targets; all four kernels): FP64 and mixed builds."""
    from paper_2411_08342_gb300 import workloads as W
    d, tg = W.wavy_torus()
    a, surf, targ = upload(ctx, d, tg, dev)
    autotune(ctx, surf, targ, 8)
    t, pm, nnz, npairs, dg = time_builds(ctx, surf, targ, dev, flush, 2, 1)
    tm, _, _, _, _ = time_builds(ctx, surf, targ, dev, flush, 1, 1, mixed=True)
    ms, mm = sum(t) / len(t), sum(tm) / len(tm)
    return {"workload": "wavy_torus_20480_p8_937k_SDSpDp", "pairs": npairs, "nnz_per_kernel": nnz,
            "fp64": {"value": 4 * nnz / (ms * 1e-3), "unit": UNIT, "ms": ms,
                     "pair_stage_tflops": flops_per_pair(8) * npairs / (sum(pm) / len(pm) * 1e-3) / 1e12},
            "mixed": {"value": 4 * nnz / (mm * 1e-3), "unit": UNIT, "ms": mm, "speedup_vs_fp64": ms / mm}}


def apply_leg(ctx, surf, targ, d, tg, dev, reps: int = 2) -> dict:
    """The corrected operator (rrq_apply: the fused kernel summing the smooth rule over all
    N_S nodes for every target and adding its CSR row) for each kernel, FP64 and mixed, on
    the FP64 corrections of this workload; kernel times by the library's CUDA events."""
    import torch
    csr = ctx.build_corrections(surf, targ, KERNELS)
    sig = torch.as_tensor(np.random.default_rng(SEED + 7).standard_normal(d.nnode), dtype=torch.float64,
                          device=dev)
    out = torch.empty(tg.n, dtype=torch.float64, device=dev)
    out32 = torch.empty_like(out)
    f64, f32, rel32 = [], [], []
    for k in KERNELS:
        for it in range(reps + 1):
            ctx.apply(surf, targ, k, csr, sig, out)
            if it > 0:
                f64.append(ctx.diagnostics()["ms_apply_smooth"])
        for it in range(reps + 1):
            ctx.apply(surf, targ, k, csr, sig, out32, mixed=True)
            if it > 0:
                f32.append(ctx.diagnostics()["ms_apply_smooth"])
        rel32.append(float((out32 - out).abs().max() / out.abs().max()))
    ctx.csr_free(csr)
    m64, m32 = statistics.median(f64), statistics.median(f32)
    return {"fp64": {"ms": m64, "interactions_per_s": tg.n * d.nnode / (m64 * 1e-3),
                     "note": "one fused kernel: dense smooth rule over all N_T x N_S pairs (the paper uses an FMM "
                             "there) plus the correction row"},
            "mixed": {"ms": m32, "interactions_per_s": tg.n * d.nnode / (m32 * 1e-3), "speedup_vs_fp64": m64 / m32,
                      "max_rel_diff_vs_fp64_apply": max(rel32),
                      "precision": "smooth terms beyond r_c in FP32 (hi/lo coordinates, compensated tile sums), "
                                   "closer ones in FP64 with the row"}}


def evaluate_leg(ctx, surf, targ, d, tg, dev, ms_build: float, reps: int = 3) -> dict:
    """Density-given near evaluation (rrq_evaluate_near, all four kernels): the correction
    applied to a density without the matrix; timed by CUDA events around the call,
    against building the four CSRs (the FP64 step time)."""
    import torch
    sig = torch.as_tensor(np.random.default_rng(SEED + 9).standard_normal(d.nnode), dtype=torch.float64, device=dev)
    outs = {k: torch.empty(tg.n, dtype=torch.float64, device=dev) for k in KERNELS}
    stream = torch.cuda.current_stream(dev)
    times = []
    for it in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.evaluate_near(surf, targ, sig, outs)
        e1.record(stream)
        e1.synchronize()
        if it > 0:
            times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    npairs = ctx.diagnostics()["npairs"]
    return {"ms": ms, "targets_per_s": tg.n / (ms * 1e-3), "pairs_per_s": npairs / (ms * 1e-3),
            "speedup_vs_matrix_build": ms_build / ms,
            "note": "S, D, S', D' corrections applied to a random density, no CSR stored"}


def stellarator_leg(ctx, dev) -> dict:
    """The stellarator of eq. stellarator (24 x 72 parameter cells, 3,456 patches, all nodes as
    targets) at p = 4 ... 14: points per second of an S-only and a D-only correction build
    (N / T with N the number of nodes, the measure of the paper's throughput table; one
    GB300 here, one CPU core there), and the relative max error of Green's identity
    1/2 u = S[du/dn] - D[u] for u = 1/|x| through rrq_apply with those two builds."""
    import torch
    from paper_2411_08342_gb300 import rrq
    from paper_2411_08342_gb300 import workloads as W
    stream = torch.cuda.current_stream(dev)
    out = {"workload": "stellarator 24x72 cells (3456 patches), on-surface nodes"}
    for p in (4, 6, 8, 10, 12, 14):
        d, tg = W.stellarator(p)
        a = rrq.device_inputs(d, tg, device=str(dev))
        surf = ctx.surface(a["order"], a["node_off"], a["xyz"], a["nrm"], a["wts"], d.ref_uv)
        targ = ctx.targets(a["txyz"], a["tnrm"], a["tself"])
        row = {"points": d.nnode}
        x = d.xyz
        r = np.linalg.norm(x, axis=1)
        u = 1.0 / r
        dudn = -np.einsum("ia,ia->i", x, d.nrm) / r ** 3
        res = {}
        for k, dens in (("S", dudn), ("D", u)):
            if p <= 8:
                ctx.csr_free(ctx.build_corrections(surf, targ, (k,)))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            csr = ctx.build_corrections(surf, targ, (k,))
            e1.record(stream)
            e1.synchronize()
            row[f"points_per_s_{k}"] = d.nnode / (e0.elapsed_time(e1) * 1e-3)
            o = torch.empty(tg.n, dtype=torch.float64, device=dev)
            ctx.apply(surf, targ, k, csr, torch.as_tensor(dens, device=dev), o)
            ctx.csr_free(csr)
            res[k] = o.cpu().numpy()
        row["green_identity_rel_err"] = float(np.abs(res["S"] - res["D"] - 0.5 * u).max() / u.max())
        out[f"p{p}"] = row
    return out


def translation_leg(ctx, dev) -> dict:
    """Step 7 both ways: the direct O(p^4) translation sums (the default) against the O(p^3)
    rotation-based translation (rrq_options.translation = 1, Sec. 2.3), FP64, all four
    kernels, on the 320-patch star with every node a target, p = 6 ... 14: device time of
    the per-pair stage (rrq_diag.ms_pairs) of one build each, after a warm-up build of each
    form on the first 64 targets."""
    from paper_2411_08342_gb300 import rrq
    from paper_2411_08342_gb300 import workloads as W
    out = {"workload": "star 320 patches, on-surface nodes, S D S' D' (FP64)"}
    for p in (6, 8, 10, 12, 14):
        d = W.discretize(W.star_surface(2), p)
        tg = W.on_surface_targets(d)
        few = W.Targets(tg.xyz[:64], tg.nrm[:64], tg.self_node[:64])
        row = {"targets": tg.n}
        for name, t in (("warm", few), ("time", tg)):
            a = rrq.device_inputs(d, t, device=str(dev))
            surf = ctx.surface(a["order"], a["node_off"], a["xyz"], a["nrm"], a["wts"], d.ref_uv)
            targ = ctx.targets(a["txyz"], a["tnrm"], a["tself"])
            for rot in (False, True):
                csr = ctx.build_corrections(surf, targ, KERNELS, rotation=rot)
                diag = ctx.diagnostics()
                ctx.csr_free(csr)
                if name == "time":
                    row["pairs"] = int(diag["npairs"])
                    row["ms_rotation" if rot else "ms_direct"] = float(diag["ms_pairs"])
        row["rotation_over_direct"] = row["ms_rotation"] / row["ms_direct"]
        out[f"p{p}"] = row
    return out


def _batch_vs_loop(ctx, dev, items) -> dict:
    """One plan over all surfaces (rrq_batch_create: near lists, CSR structure, autotuned
    launch shapes, value computation recorded as one CUDA graph), executed after one
    warm-up execution, FP64 and mixed; against building the same surfaces one by one with
    rrq_build_corrections (FP64 and mixed, the shapes the batch tuned).  Device times by
    CUDA events; the one-by-one loop after one warm-up pass."""
    import torch
    from paper_2411_08342_gb300 import rrq
    arrs = [rrq.device_inputs(d, tg, device=str(dev)) for d, tg in items]
    surfs = [ctx.surface(a["order"], a["node_off"], a["xyz"], a["nrm"], a["wts"], d.ref_uv)
             for a, (d, _) in zip(arrs, items)]
    targs = [ctx.targets(a["txyz"], a["tnrm"], a["tself"]) for a in arrs]
    orders = sorted({int(d.p) for d, _ in items})
    out = {"surfaces": len(items), "targets": int(sum(tg.n for _, tg in items)),
           "patches": int(sum(d.npatch for d, _ in items))}
    entries = 0
    for mixed in (False, True):
        b = ctx.batch(surfs, targs, mixed=mixed, autotune=True)
        b.execute()
        b.execute()
        ms = ctx.diagnostics()["ms_pairs"]
        info = b.info()
        entries = info["nnz"] * len(KERNELS)
        out["mixed" if mixed else "fp64"] = {
            "value": entries / (ms * 1e-3), "unit": UNIT, "ms_execute": ms, "ms_create": info["ms_create"],
            "ms_autotune": info["ms_autotune"], "graph_kernels": info["graph_kernels"],
            "tile": {p: info["tile"][p] for p in orders}, "persistent": {p: info["persistent"][p] for p in orders}}
        out["pairs"] = info["npairs"]
        out["nnz_per_kernel"] = info["nnz"]
        b.close()
    for mixed in (False, True):
        stream = torch.cuda.current_stream(dev)
        for it in range(1):
            torch.cuda.synchronize(dev)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            for sf, tg in zip(surfs, targs):
                ctx.csr_free(ctx.build_corrections(sf, tg, KERNELS, mixed=mixed))
            ev1.record(stream)
            ev1.synchronize()
        ms_loop = ev0.elapsed_time(ev1)
        out["one_by_one_mixed" if mixed else "one_by_one_fp64"] = {"value": entries / (ms_loop * 1e-3), "unit": UNIT,
                                                                   "ms": ms_loop}
    out["batched_vs_one_by_one_fp64"] = out["fp64"]["value"] / out["one_by_one_fp64"]["value"]
    out["batched_vs_one_by_one_mixed"] = out["mixed"]["value"] / out["one_by_one_mixed"]["value"]
    out["speedup_batched_mixed_vs_one_by_one_fp64"] = out["mixed"]["value"] / out["one_by_one_fp64"]["value"]
    return out


def batched_leg(ctx, dev) -> dict:
    """The batching pattern on two workloads: the 64 seeded star surfaces of 80..5120
    patches (p in {4, 6, 8}, all on-surface nodes as targets), and 256 small ones (80 or 320
    patches), where one launch per surface and order would leave most of the GPU idle."""
    from paper_2411_08342_gb300 import workloads as W
    big = _batch_vs_loop(ctx, dev, W.star_batch())
    big["workload"] = "star_batch64 (80..5120 patches, p in {4,6,8}, on-surface nodes)"
    small = _batch_vs_loop(ctx, dev, W.star_batch(256, levels=(1, 2), seed=SEED + 11))
    small["workload"] = "star_batch256 small (80 or 320 patches, p in {4,6,8}, on-surface nodes)"
    big["small_surfaces"] = small
    return big


def measured_peaks() -> dict:
    """The measured peaks of the GB300s (MEASURED_PEAKS.json, written by the
    machine's owner), else the fallback of one earlier measurement (6.8 TB/s HBM copy,
    1.9 PFLOP/s bf16), marked as such."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
            d.setdefault("source", "measured")
            return d
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


def e2e_leg(ctx, d, tg, nnz, dev, flush, args, world, total_entries):
    """Same metric through the C ABI with host buffers: pinned inputs copied in, and the
    four CSRs written by the per-pair kernels straight into pinned host memory
    (rrq_build_corrections_into), all inside the timed region (two builds, after the
    device-resident ones)."""
    import torch
    host = {k: np.ascontiguousarray(v) for k, v in dict(order=d.order, node_off=d.node_off, xyz=d.xyz, nrm=d.nrm,
                                                         wts=d.wts, txyz=tg.xyz, tnrm=tg.nrm,
                                                         tself=tg.self_node).items()}
    pin = {k: torch.from_numpy(v).pin_memory().numpy() for k, v in host.items()}
    hsurf = ctx.surface(pin["order"], pin["node_off"], pin["xyz"], pin["nrm"], pin["wts"], d.ref_uv)
    htarg = ctx.targets(pin["txyz"], pin["tnrm"], pin["tself"])
    out_rowptr = torch.empty(tg.n + 1, dtype=torch.int64, pin_memory=True).numpy()
    out_col = torch.empty(nnz, dtype=torch.int32, pin_memory=True).numpy()
    out_vals = {k: torch.empty(nnz, dtype=torch.float64, pin_memory=True).numpy() for k in KERNELS}
    h2d = sum(v.nbytes for v in pin.values())
    d2h = out_rowptr.nbytes + out_col.nbytes + sum(v.nbytes for v in out_vals.values())
    times = []
    for it in range(2):
        flush.fill_(1.0)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ctx.build_corrections_into(hsurf, htarg, out_rowptr, out_col, out_vals, KERNELS, inputs_on_host=True)
        torch.cuda.synchronize(dev)
        times.append(time.perf_counter() - t0)
    e2e_s = reduce_max(sum(times) / len(times), world, dev)
    return {"value": total_entries / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "steps": len(times), "api": "rrq_build_corrections_into (kernels write pinned host memory)"}


def cpu_baseline(ntarg_sample: int) -> dict:
    """The oracle, as it stands, on a bounded sample of the headline workload (the first
    ntarg_sample targets, all their near pairs, all four kernels), on all host cores; and
    on one core (as the paper measures) on a 16x smaller sample."""
    from oracle import oracle as O
    d, tg = workload()
    sel = np.arange(min(ntarg_sample, tg.n))
    osf = O.OracleSurface(d)
    t0 = time.perf_counter()
    rowptr, col, vals, _ = osf.csr_rows(tg, sel, KERNELS)
    dt = time.perf_counter() - t0
    entries = float(rowptr[-1]) * len(KERNELS)
    cores = len(os.sched_getaffinity(0))
    threads = int(os.environ.get("OMP_NUM_THREADS", cores))
    out = {"value": entries / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"first {len(sel)} of the {tg.n} targets, all near pairs, 4 kernels ({int(entries)} entries, "
                     f"{dt:.1f} s)", "seconds": dt}
    try:
        import ctypes
        gomp = ctypes.CDLL("libgomp.so.1")
        gomp.omp_set_num_threads(1)
        sel1 = np.arange(max(1, len(sel) // 16))
        t0 = time.perf_counter()
        rp1, _, _, _ = osf.csr_rows(tg, sel1, KERNELS)
        dt1 = time.perf_counter() - t0
        gomp.omp_set_num_threads(threads)
        e1 = float(rp1[-1]) * len(KERNELS)
        out["one_core"] = {"value": e1 / dt1, "unit": UNIT, "points_per_s": len(sel1) / dt1,
                           "sample": f"first {len(sel1)} targets ({int(e1)} entries, {dt1:.1f} s)"}
    except OSError:
        out["one_core"] = None
    return out


def bench_reference(args):
    """The reference arm: the CPU oracle as it stands, on all host cores, each step a
    bounded sample (args.cpu_targets consecutive targets) of the headline workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    d, tg = workload()
    osf = O.OracleSurface(d)
    n = args.ref_targets
    times, entries = [], 0.0
    for it in range(args.warmup + args.steps):
        sel = np.arange(it * n, (it + 1) * n) % tg.n
        t0 = time.perf_counter()
        rowptr, _, _, _ = osf.csr_rows(tg, sel, KERNELS)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
            entries += float(rowptr[-1]) * len(KERNELS)
    tot = sum(times)
    value = entries / tot
    cores = int(os.environ.get("OMP_NUM_THREADS", len(os.sched_getaffinity(0))))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_targets_per_step": n},
            "impl": "reference",
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value, "unit": UNIT,
                             "sample": f"{n} consecutive targets of the {tg.n} per step, all near pairs, 4 kernels"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-targets", type=int, default=20000, help="targets of the CPU-baseline sample")
    ap.add_argument("--ref-targets", type=int, default=8000,
                    help="targets per step of the reference arm (the oracle on the host cores)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-apply", action="store_true", help="skip the apply, SpMV and evaluation timings")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-surface batch and the stellarator")
    ap.add_argument("--no-extra", action="store_true", help="skip the star and torus workloads")
    ap.add_argument("--no-autotune", action="store_true", help="default launch shapes (for profiling captures)")
    ap.add_argument("--levels", type=int, default=6,
                    help="ellipsoid mesh levels: 20 * 4^levels patches (6 = the 81,920-patch workload)")
    args = ap.parse_args()
    if args.impl == "reference":
        bench_reference(args)
    else:
        bench_gpu(args)


if __name__ == "__main__":
    main()
