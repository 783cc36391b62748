"""Benchmark: near-field correction entries per second on one GB300.

Workload (one step = one full correction build, all four kernels S, D, S', D'):
star-shaped surface r = 1 + 0.2 Re Y_3^2 + 0.1 Re Y_5^1 on a 1280-patch icosahedral
mesh, order p = 6 (21 nodes per patch, 26,880 nodes), 200,000 off-surface targets at
distance 10^-k h (k ~ U[0,6]) along the normal of a random patch.  Inputs are seeded
and synthetic.  The timed region starts with geometry and targets resident in device
memory and ends with the four CSR matrices resident in device memory: near list,
per-patch precompute, pair kernel, CSR assembly.  An L2 flush (a 512 MB write) runs
between timed steps, outside the timed region.

Output: one JSON line (rank 0).  `--impl reference` times the CPU oracle instead, on a
bounded sample of the same workload.  With torchrun (N > 1) every rank builds its own
seeded 200k-target set against the same surface (weak scaling, no collective in the
data path); the step time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
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

METRIC = "near-correction entries/s at 1e-10 rel err (FP64)"
UNIT = "entries/s"
WORKLOAD = "star1280_p6_200k_offsurface_SDSpDp"
NTARG = 200_000
P = 6
KERNELS = ("S", "D", "SP", "DP")
SEED = 20241115


def workload(rank: int = 0, ntarg: int = NTARG):
    from paper_2411_08342_gb300 import workloads as W
    return W.star1280(P, ntarg, seed=SEED + 1000 * rank)


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
    # Step 6: V (3 FMA x complex) for j >= 1; Q (18 FMA) and dQ/dnu' (24 FMA) for j >= 2
    line = ns * (12 * n1 + 36 * n2 + 48 * n2)
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


def bench_gpu(args):
    import torch

    from paper_2411_08342_gb300 import rrq
    rank, world, lrank = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", lrank))
    torch.cuda.set_device(lrank)
    dev = torch.device("cuda", lrank)
    d, tg = workload(rank, args.ntarg)
    ctx = rrq.Context(lrank)
    arrs = rrq.device_inputs(d, tg, device=str(dev))
    surf = ctx.surface(arrs["order"], arrs["node_off"], arrs["xyz"], arrs["nrm"], arrs["wts"], d.ref_uv)
    targ = ctx.targets(arrs["txyz"], arrs["tnrm"], arrs["tself"])
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    # one-time autotuning of the per-pair launch shapes on this problem (kept in the context)
    tuned = {}
    for m in (False, True):
        b = ctx.batch([surf], [targ], KERNELS, mixed=m, autotune=True)
        info = b.info()
        b.close()
        tuned["mixed" if m else "fp64"] = {"tile": info["tile"][P], "persistent": info["persistent"][P],
                                           "ms_autotune": info["ms_autotune"]}

    def step(mixed=False):
        csr = ctx.build_corrections(surf, targ, KERNELS, mixed=mixed)
        nnz, npairs = csr.nnz, csr.npairs
        ctx.csr_free(csr)
        return nnz, npairs

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(lrank)
    clocks.start()
    time.sleep(0.3)
    times, pair_ms, nnz, npairs = [], [], 0, 0
    torch.cuda.synchronize(dev)
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        nnz, npairs = step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        pair_ms.append(ctx.diagnostics()["ms_pairs"])
    torch.cuda.synchronize(dev)
    diag = ctx.diagnostics()           # stage times and launch count of the last FP64 build
    if world > 1:
        torch.distributed.barrier()
    # the mixed-precision build (line integrals in double-float FP32) on the same inputs
    mtimes = []
    for it in range(args.steps + 1):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(mixed=True)
        e1.record(stream)
        e1.synchronize()
        if it > 0:
            mtimes.append(e0.elapsed_time(e1))
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    mdiag = ctx.diagnostics()
    ms_step = reduce_max(sum(times) / len(times), world, dev)
    entries = nnz * len(KERNELS)
    total_entries = reduce_sum(float(entries), world, dev)
    value = total_entries / (ms_step * 1e-3)
    ms_mixed = reduce_max(sum(mtimes) / len(mtimes), world, dev)

    # e2e: host buffers through the C ABI (H2D of inputs and D2H of the four CSRs timed)
    e2e = None
    if args.no_e2e:
        host = None
    else:
        e2e = e2e_leg(ctx, d, tg, nnz, dev, flush, args, world, total_entries)
    # roofline of the dominant kernel (the per-pair kernel), FP64 ALU bound.  DRAM traffic of
    # k_pairs_tile<6, false, 5> on this workload from a one-pass ncu capture
    # (dram__bytes_read.sum + dram__bytes_write.sum); None once the kernel changes.
    traffic = 2_131_227_136 + 3_820_670_208
    peak = ctx.fma_peak_tflops(fp32=False)
    peak32 = ctx.fma_peak_tflops(fp32=True)
    fpp = flops_per_pair(P)
    pair_s = sum(pair_ms) / len(pair_ms) * 1e-3
    achieved = fpp * npairs / pair_s / 1e12
    # kernel launches per step: per-order precompute and pair kernels, near list, scans, items
    launches = diag.get("kernel_launches", None)
    apply = None if args.no_apply else apply_leg(ctx, surf, targ, d, tg, dev)
    evaluate = None if args.no_apply else evaluate_leg(ctx, surf, targ, d, tg, dev, ms_step)
    batched = None if (args.no_batched or world > 1) else batched_leg(ctx, dev)
    stell = None if (args.no_batched or world > 1) else stellarator_leg(ctx, dev)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded star surface and off-surface targets)",
        "config": {"workload": WORKLOAD, "patches": d.npatch, "p": P, "nodes": d.nnode, "targets": tg.n,
                   "kernels": list(KERNELS), "pairs": npairs, "nnz_per_kernel": nnz,
                   "l2": "512 MB flush between timed steps", "parallelism": f"weak x{world}"},
        "e2e": e2e,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": traffic, "traffic_note": "bytes per launch of k_pairs_tile<6, false, 5> (the autotuned FP64 shape), one-pass ncu capture",
                     "kernel": "k_roots<6> + k_uside<6> + k_pairs_tile<6, false, T> (one per-pair stage)",
                     "peak_note": "measured FP64 FMA peak (rrq_measure_fma_peak); FP32 FMA peak %.1f TFLOP/s" % peak32,
                     "flops_per_pair": fpp, "kernel_ms": pair_s * 1e3},
        "stage_ms": {"precompute": diag["ms_precompute"], "near_and_items": diag["ms_near"], "pairs": diag["ms_pairs"]},
        "fit_kappa_max": diag["kappa_max"],
        "launch_shape": tuned,
        "clocks": clk,
        "gpu_launches": launches * args.steps if launches is not None else None,
        "points_per_s": world * tg.n / (ms_step * 1e-3),
        "apply": apply,
        "evaluate_near": evaluate,
        "batched": batched,
        "stellarator": stell,
        "mixed": {"value": total_entries / (ms_mixed * 1e-3), "unit": UNIT, "ms_per_step": ms_mixed,
                  "stage_ms": {"precompute": mdiag["ms_precompute"], "near_and_items": mdiag["ms_near"],
                               "pairs": mdiag["ms_pairs"]},
                  "speedup_vs_fp64": ms_step / ms_mixed,
                  "precision": "line integrals, translations and fit contraction in double-float FP32 "
                               "(about 48 bits); roots, recurrences, Omega_0, harmonics, smooth rule FP64",
                  "parity": "apply-level error as FP64; rows within 32x the oracle's own rounding sensitivity "
                            "(tests/test_gpu_mixed.py)"},
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_targets)
        line["cpu_baseline"]["value"] = line["cpu_baseline"]["entries_per_s"]
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def apply_leg(ctx, surf, targ, d, tg, dev, reps: int = 3) -> dict:
    """The apply (y = smooth direct sum + CSR correction times sigma) for each kernel on
    the FP64 corrections of this workload, timed per device kernel by the library's own
    CUDA events: SpMV against the measured HBM copy bandwidth, the direct sum in
    interactions/s.  The CSR (about 1.1 GB per kernel) is larger than L2."""
    import torch
    csr = ctx.build_corrections(surf, targ, KERNELS)
    nnz = csr.nnz
    sig = torch.as_tensor(np.random.default_rng(SEED + 7).standard_normal(d.nnode), dtype=torch.float64,
                          device=dev)
    out = torch.empty(tg.n, dtype=torch.float64, device=dev)
    out32 = torch.empty_like(out)
    spmv, smooth, smooth32, spmv32, rel32 = [], [], [], [], []
    for k in KERNELS:
        for it in range(reps + 1):
            ctx.apply(surf, targ, k, csr, sig, out)
            dg = ctx.diagnostics()
            if it > 0:
                spmv.append(dg["ms_apply_spmv"])
                smooth.append(dg["ms_apply_smooth"])
        for it in range(reps + 1):
            ctx.apply(surf, targ, k, csr, sig, out32, mixed=True)
            if it > 0:
                dg = ctx.diagnostics()
                smooth32.append(dg["ms_apply_smooth"])
                spmv32.append(dg["ms_apply_spmv"])
        rel32.append(float((out32 - out).abs().max() / out.abs().max()))
    ctx.csr_free(csr)
    ms_spmv = statistics.median(spmv)
    ms_smooth = statistics.median(smooth)
    ms_smooth32 = statistics.median(smooth32)
    # algorithmic bytes of one SpMV: val (8) + col (4) per entry, rowptr, out read + write, sigma
    spmv_bytes = nnz * 12 + (tg.n + 1) * 8 + tg.n * 16 + d.nnode * 8
    peak = measured_peaks().get("hbm_gbs")
    gbs = spmv_bytes / (ms_spmv * 1e-3) / 1e9
    return {"spmv": {"ms": ms_spmv, "nnz": nnz, "bytes": spmv_bytes, "achieved_gbs": gbs, "peak_gbs": peak,
                     "frac": gbs / peak if peak else None, "peak_note": "of measured HBM copy bandwidth"},
            "direct_sum": {"ms": ms_smooth, "interactions_per_s": tg.n * d.nnode / (ms_smooth * 1e-3),
                           "note": "dense smooth rule over all N_T x N_S pairs (the paper uses an FMM here)"},
            "apply_mixed": {"ms_far_fp32": ms_smooth32, "ms_spmv_near_fp64": statistics.median(spmv32),
                            "interactions_per_s": tg.n * d.nnode / ((ms_smooth32 + statistics.median(spmv32)) * 1e-3),
                            "speedup_vs_fp64": (ms_smooth + ms_spmv) / (ms_smooth32 + statistics.median(spmv32)),
                            "max_rel_diff_vs_fp64_apply": max(rel32),
                            "precision": "smooth terms beyond r_c in FP32 (hi/lo coordinates, compensated tile "
                                         "sums), closer ones in FP64 inside the correction SpMV"}}


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
    targets) at p = 4, 6, 8, 10, 12: points per second of an S-only and a D-only correction build
    (N / T with N the number of nodes, the measure of the paper's throughput table; one
    GB300 here, one CPU core there), and the relative max error of Green's identity
    1/2 u = S[du/dn] - D[u] for u = 1/|x| through rrq_apply."""
    import torch
    from paper_2411_08342_gb300 import rrq
    from paper_2411_08342_gb300 import workloads as W
    stream = torch.cuda.current_stream(dev)
    out = {"workload": "stellarator 24x72 cells (3456 patches), on-surface nodes"}
    for p in (4, 6, 8, 10, 12):
        d, tg = W.stellarator(p)
        a = rrq.device_inputs(d, tg, device=str(dev))
        surf = ctx.surface(a["order"], a["node_off"], a["xyz"], a["nrm"], a["wts"], d.ref_uv)
        targ = ctx.targets(a["txyz"], a["tnrm"], a["tself"])
        row = {"points": d.nnode}
        for k in ("S", "D"):
            times = []
            for it in range(3 if p <= 8 else 2):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                csr = ctx.build_corrections(surf, targ, (k,))
                e1.record(stream)
                e1.synchronize()
                ctx.csr_free(csr)
                if it > 0:
                    times.append(e0.elapsed_time(e1))
            row[f"points_per_s_{k}"] = d.nnode / (min(times) * 1e-3)
        x = d.xyz
        r = np.linalg.norm(x, axis=1)
        u = 1.0 / r
        dudn = -np.einsum("ia,ia->i", x, d.nrm) / r ** 3
        csr = ctx.build_corrections(surf, targ, ("S", "D"))
        oS = torch.empty(tg.n, dtype=torch.float64, device=dev)
        oD = torch.empty_like(oS)
        ctx.apply(surf, targ, "S", csr, torch.as_tensor(dudn, device=dev), oS)
        ctx.apply(surf, targ, "D", csr, torch.as_tensor(u, device=dev), oD)
        ctx.csr_free(csr)
        row["green_identity_rel_err"] = float(np.abs((oS - oD).cpu().numpy() - 0.5 * u).max() / u.max())
        out[f"p{p}"] = row
    return out


def batched_leg(ctx, dev) -> dict:
    """The batched form: 64 seeded star surfaces (80..5120 patches, p in {4, 6, 8}, all
    on-surface nodes as targets) in one plan (rrq_batch_create: near lists, CSR structure,
    autotuned launch shapes, value computation recorded as one CUDA graph), executed
    after one warm-up execution, FP64 and mixed; against building the same surfaces one
    by one with rrq_build_corrections in FP64.  Device times by CUDA events."""
    import torch
    from paper_2411_08342_gb300 import rrq
    from paper_2411_08342_gb300 import workloads as W
    items = W.star_batch()
    arrs = [rrq.device_inputs(d, tg, device=str(dev)) for d, tg in items]
    surfs = [ctx.surface(a["order"], a["node_off"], a["xyz"], a["nrm"], a["wts"], d.ref_uv)
             for a, (d, _) in zip(arrs, items)]
    targs = [ctx.targets(a["txyz"], a["tnrm"], a["tself"]) for a in arrs]
    out = {"workload": "star_batch64 (80..5120 patches, p in {4,6,8}, on-surface nodes)",
           "surfaces": len(items), "targets": int(sum(tg.n for _, tg in items))}
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
            "tile": {p: info["tile"][p] for p in (4, 6, 8)},
            "persistent": {p: info["persistent"][p] for p in (4, 6, 8)}}
        out["pairs"] = info["npairs"]
        out["nnz_per_kernel"] = info["nnz"]
        b.close()
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(torch.cuda.current_stream(dev))
    for sf, tg in zip(surfs, targs):
        ctx.csr_free(ctx.build_corrections(sf, tg, KERNELS))
    ev1.record(torch.cuda.current_stream(dev))
    ev1.synchronize()
    ms_loop = ev0.elapsed_time(ev1)
    out["one_by_one_fp64"] = {"value": entries / (ms_loop * 1e-3), "unit": UNIT, "ms": ms_loop}
    out["speedup_batched_mixed_vs_one_by_one_fp64"] = out["mixed"]["value"] / out["one_by_one_fp64"]["value"]
    return out


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def e2e_leg(ctx, d, tg, nnz, dev, flush, args, world, total_entries):
    """Same metric through the C ABI with host buffers: pinned inputs copied in, and the
    four CSRs written by the per-pair kernels straight into pinned host memory
    (rrq_build_corrections_into), all inside the timed region.  For comparison, the
    same through rrq_build_corrections followed by rrq_csr_copy to the host."""
    import torch
    host = {k: np.ascontiguousarray(v) for k, v in dict(order=d.order, node_off=d.node_off, xyz=d.xyz, nrm=d.nrm,
                                                         wts=d.wts, txyz=tg.xyz, tnrm=tg.nrm,
                                                         tself=tg.self_node).items()}
    pin = {k: torch.from_numpy(v).pin_memory().numpy() for k, v in host.items()}
    hsurf = ctx.surface(pin["order"], pin["node_off"], pin["xyz"], pin["nrm"], pin["wts"], d.ref_uv)
    htarg = ctx.targets(pin["txyz"], pin["tnrm"], pin["tself"])
    out_rowptr = torch.empty(tg.n + 1, dtype=torch.int64).pin_memory().numpy()
    out_col = torch.empty(nnz, dtype=torch.int32).pin_memory().numpy()
    out_vals = {k: torch.empty(nnz, dtype=torch.float64).pin_memory().numpy() for k in KERNELS}
    h2d = sum(v.nbytes for v in pin.values())
    d2h = out_rowptr.nbytes + out_col.nbytes + sum(v.nbytes for v in out_vals.values())
    times, copied = [], []
    for it in range(max(2, args.steps // 2) + 1):
        flush.fill_(1.0)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ctx.build_corrections_into(hsurf, htarg, out_rowptr, out_col, out_vals, KERNELS, inputs_on_host=True)
        torch.cuda.synchronize(dev)
        if it > 0:
            times.append(time.perf_counter() - t0)
    for it in range(2):
        flush.fill_(1.0)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        csr = ctx.build_corrections(hsurf, htarg, KERNELS, inputs_on_host=True)
        t1 = time.perf_counter()
        ctx.csr_to_host(csr, KERNELS, out=(out_rowptr, out_col, out_vals))
        t2 = time.perf_counter()
        ctx.csr_free(csr)
        torch.cuda.synchronize(dev)
        if it > 0:
            copied.append((time.perf_counter() - t0, t1 - t0, t2 - t1))
    e2e_s = reduce_max(sum(times) / len(times), world, dev)
    return {"value": total_entries / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "api": "rrq_build_corrections_into (kernels write pinned host memory)",
            "build_then_copy": {"value": total_entries / copied[0][0], "ms_build": 1e3 * copied[0][1],
                                "ms_copy_to_host": 1e3 * copied[0][2],
                                "api": "rrq_build_corrections + rrq_csr_copy"}}


def cpu_baseline(ntarg_sample: int) -> dict:
    """The oracle, as it stands, on a bounded sample of the same workload (the first
    ntarg_sample targets, all their near pairs, all four kernels), on all host cores."""
    from oracle import oracle as O
    d, tg = workload(0)
    sel = np.arange(min(ntarg_sample, tg.n))
    osf = O.OracleSurface(d)
    t0 = time.perf_counter()
    rowptr, col, vals, _ = osf.csr_rows(tg, sel, KERNELS)
    dt = time.perf_counter() - t0
    entries = float(rowptr[-1]) * len(KERNELS)
    cores = len(os.sched_getaffinity(0))
    threads = int(os.environ.get("OMP_NUM_THREADS", cores))
    out = {"entries_per_s": entries / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"first {len(sel)} of the 200k targets, all near pairs, 4 kernels ({int(entries)} entries, "
                     f"{dt:.1f} s)", "seconds": dt}
    # one core, as the paper measures (its own Fortran on one EPYC core): a 16x smaller sample
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
        out["one_core"] = {"entries_per_s": e1 / dt1, "points_per_s": len(sel1) / dt1,
                           "sample": f"first {len(sel1)} targets ({int(e1)} entries, {dt1:.1f} s)"}
    except OSError:
        out["one_core"] = None
    return out


def bench_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    d, tg = workload(0)
    osf = O.OracleSurface(d)
    n = args.cpu_targets
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
                             "sample": f"{n} consecutive targets of the 200k per step, all near pairs, 4 kernels"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-targets", type=int, default=40000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-apply", action="store_true", help="skip the apply (SpMV + direct sum) timing")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-surface batched build")
    ap.add_argument("--ntarg", type=int, default=NTARG, help="targets per rank (default: the workload's 200k)")
    args = ap.parse_args()
    if args.impl == "reference":
        bench_reference(args)
    else:
        bench_gpu(args)


if __name__ == "__main__":
    main()
