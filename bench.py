"""Benchmark of the matchgate-shadow overlap hot path on GB300.

One step = one pass of the hot path over one batch: build the device snapshot
set from (Q, b) (qcs_build_snapshots) and evaluate the shadow overlaps of all
walkers against all snapshots (qcs_overlap), FP64, at the paper-shaped size
n = 16 modes, ne = 8 electrons, 1024 walkers x 20000 snapshots (Haar Q,
uniform 16-bit b, seed 0).  The metric is walker x snapshot pairs per second
(every pair of the batch counts, including the parity -1 pairs, which are
exactly zero and skipped).

Printed JSON line (rank 0):
  value          device-resident throughput (inputs in HBM before the timed region)
  e2e            the same through the C ABI from pinned HOST buffers: copies of Q, b
                 and the walkers in, overlaps out, inside the timed region
  roofline       dominant kernel (pair_overlap_kernel) against the FP64 ALU peak
  cpu_baseline   the CPU oracle on a bounded sample of the same workload
  clocks         nvidia-smi samples taken during the timed region

--impl reference times the CPU oracle instead (the reference arm of this
benchmark).  Under torchrun each rank runs the full workload on its own GPU
(independent replicas, no collective in the data path); the time is the
maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "walker×snapshot overlap(+grad) pairs/s at n=16; % of FP64 peak vs plain GPU path"
# FP64 ALU peak of a GB300 from unit counts: 152 SMs x 4 FP64 flop/clk/SM x 2.07 GHz
# maximum SM clock.  The sustained rate of register-only FMA chains is measured in
# each run on the same GPU (qcs_fp64_fma_rate) and reported beside every FP64 roofline.
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12
L2_FLUSH_BYTES = 256 << 20


def measured_peaks() -> dict:
    """The machine's measured peaks (MEASURED_PEAKS.json at the repository root), else the
    fallback figures of one earlier GB300 measurement (HBM 6.8 TB/s, BF16 1.9 PFLOP/s burst,
    1.7 sustained), marked as such."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        d["source"] = "measured"
        return d
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


def add_dfma_context(obj, rate):
    """Beside every FP64 ("alu") roofline, the fraction of the measured FMA rate."""
    if isinstance(obj, dict):
        if obj.get("bound") == "alu" and isinstance(obj.get("achieved"), float):
            obj["dfma_probe"] = {"tflops": rate, "frac": obj["achieved"] / rate,
                                 "source": "register-only FP64 FMA chains on this GPU in this run "
                                           "(qcs_fp64_fma_rate)"}
        for v in list(obj.values()):
            add_dfma_context(v, rate)
    elif isinstance(obj, list):
        for v in obj:
            add_dfma_context(v, rate)


def max_over_ranks(t: float, ws: int) -> float:
    """Largest of a per-rank time over all ranks (the whole job ends with the slowest rank)."""
    if ws <= 1:
        return t
    import torch
    import torch.distributed as dist

    tt = torch.tensor([t], dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"qcs_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


CSRC = os.path.join(ROOT, "paper_2506_22408_gb300", "csrc")
# Source files each timed kernel is compiled from; the committed DRAM figure of a
# kernel is used only while all of them are unchanged.
KERNEL_SOURCES = {
    "tc_pair_kernel": ["qcs_tcpair.cu", "qcs_ozaki.cuh", "qcs_tc.cuh", "qcs_pair.cuh", "qcs_common.cuh"],
    "pair_overlap_kernel": ["qcs_overlap.cu", "qcs_group.cuh", "qcs_pair.cuh", "qcs_common.cuh"],
    "split_pair_kernel": ["qcs_split.cu", "qcs_pair.cuh", "qcs_tc.cuh", "qcs_common.cuh"],
    "grad_pair_kernel": ["qcs_grad.cu", "qcs_group.cuh", "qcs_pair.cuh", "qcs_common.cuh"],
    "rdm_syrk_kernel": ["qcs_rdm.cu"],
    "energy_pair_kernel": ["qcs_energy.cu", "qcs_group.cuh", "qcs_pair.cuh", "qcs_common.cuh"],
    # the FP64 ALU pair kernel in its batched launch over the five systems of the batching
    # workload (a record of its own: another workload)
    "pair_overlap_kernel_batched": ["qcs_overlap.cu", "qcs_group.cuh", "qcs_pair.cuh", "qcs_common.cuh"],
}

# workload name of the batched launch's traffic record
BATCH_WORKLOAD = "batch n=8,12,16,20,24 ne=n/2, 1024/512/256/128/64 walkers, 2000/5000/10000/20000/40000 snapshots"


def kernel_source_sha(kernel: str) -> str:
    """Hash of the kernel's sources with comments and blank space removed, so that a
    traffic record stays valid across comment edits and lapses with any code change."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        src = open(os.path.join(CSRC, f), encoding="utf-8").read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()


def traffic_for(kernel: str, workload: str):
    """DRAM bytes per launch (read + write) from the committed ncu record, if it was
    taken on the current sources and on this workload; else None."""
    path = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        r = json.load(open(path)).get(kernel)
        if r and r.get("source_sha256") == kernel_source_sha(kernel) and r.get("workload") == workload:
            return r.get("bytes_per_launch")
    except Exception:
        return None
    return None


def run_e2e(args, data, dev, step, barrier, ws, wl):
    """Same metric through the C ABI from pinned HOST buffers: H2D copies of Q, b and
    the walkers and the D2H copy of the overlaps are inside the timed region."""
    import torch
    import torch.distributed as dist

    hQ = torch.from_numpy(data["Q"]).pin_memory()
    hb = torch.from_numpy(data["b"]).pin_memory()
    hP = torch.from_numpy(data["Phi"]).pin_memory()
    hO = torch.empty(wl.W, dtype=torch.complex128).pin_memory()
    e2e_steps = max(3, min(args.steps, 5))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        Q = hQ.to(dev, non_blocking=True)
        b = hb.to(dev, non_blocking=True)
        Phi = hP.to(dev, non_blocking=True)
        snaps, ov = step(Q, b, Phi)
        hO.copy_(ov, non_blocking=True)
        torch.cuda.synchronize()
        del snaps
    t_e2e = time.perf_counter() - t0
    t_e2e = max_over_ranks(t_e2e, ws)
    h2d = hQ.numel() * 8 + hb.numel() + hP.numel() * 16
    d2h = hO.numel() * 16
    return {"value": ws * wl.W * wl.P * e2e_steps / t_e2e, "unit": "pairs/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "steps": e2e_steps}


def run_grad(args, ctx, dev, barrier, ws):
    """Differentiation workload: n = 16, ne = 8, 512 walkers x 10000 snapshots; one
    step = snapshot build + overlaps and holomorphic gradients (qcs_overlap_grad) +
    force bias over 64 Cholesky vectors (qcs_force_bias)."""
    import torch
    import torch.distributed as dist

    from paper_2506_22408_gb300 import qcs, synth

    wl = synth.DIFFERENTIATION
    if args.grad_walkers or args.grad_snapshots:
        import dataclasses

        W, P = args.grad_walkers or wl.W, args.grad_snapshots or wl.P
        wl = dataclasses.replace(wl, name=f"n={wl.n} ne={wl.ne} {W}x{P} nchol={wl.nchol} (reduced profiling case)",
                                 W=W, P=P)
    data = wl.generate(seed=0)
    Q = torch.from_numpy(data["Q"]).to(dev)
    b = torch.from_numpy(data["b"]).to(dev)
    Phi = torch.from_numpy(data["Phi"]).to(dev)
    L = torch.from_numpy(data["L"].astype(np.complex128)).to(dev)

    def step():
        snaps = qcs.Snapshots(ctx, Q, b)
        ov, g = qcs.overlap_grad(ctx, snaps, Phi)
        xb = qcs.force_bias(ctx, L, Phi, ov, g, sqrt_dt=0.1)
        return snaps, xb

    snaps, _ = step()
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    npar = int((snaps.parity() == 1).sum().item())
    del snaps
    steps = max(2, min(args.steps, 3))
    ctx.profile(True)
    ctx.profile_read()
    barrier()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        snaps, xb = step()
    e1.record(stream)
    barrier()
    ctx.profile(False)
    kms, kl = ctx.profile_read()
    t = e0.elapsed_time(e1) / 1e3
    t = max_over_ranks(t, ws)
    fpp = qcs.grad_flops_per_pair(wl.n, wl.ne)
    avg = kms / max(kl, 1)
    ach = fpp * npar * wl.W / (avg * 1e-3) / 1e12
    return {"metric": "walker x snapshot overlap+grad pairs/s (with force bias)", "value": ws * wl.W * wl.P * steps / t,
            "unit": "pairs/s", "ms_per_step": 1e3 * t / steps, "steps": steps,
            "config": {"workload": wl.name + " (Haar Q, uniform b, seed 0)", "parity_plus_snapshots": npar,
                       "nchol": wl.nchol},
            "roofline": {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": ach / FP64_PEAK_TFLOPS, "traffic": traffic_for("grad_pair_kernel", wl.name),
                         "kernel": "grad_pair_kernel", "kernel_ms": avg, "flops_per_launch": fpp * npar * wl.W},
            "gpu_launches_per_step": 6}


def run_batch(args, ctx, dev, barrier, ws):
    """Batching workload: five active spaces n = 8, 12, 16, 20, 24 (ne = n/2) with
    1024/512/256/128/64 walkers and 2000/5000/10000/20000/40000 snapshots.  One AFQMC
    step = a stand-in propagation of every system's walkers (walkers <- U walkers with a
    fixed small unitary U = exp(eps K) per system, cuBLAS through torch) followed by ONE
    qcs_overlap_batched call (one persistent pair-kernel launch over all systems);
    --batch-steps steps are captured in one CUDA graph, which is replayed."""
    import dataclasses

    import torch
    import torch.distributed as dist

    from paper_2506_22408_gb300 import qcs, synth

    rng = np.random.default_rng(7)
    systems, Us, outs, tuned = [], [], [], []
    for wl0 in synth.BATCH_SYSTEMS:
        wl = dataclasses.replace(wl0, W=max(1, int(round(wl0.W * args.batch_walker_scale))))
        d = wl.generate(seed=0)
        # the batched launch runs the FP64 ALU pair kernel: tune that path for each system
        tuned.append(ctx.autotune(wl.n, wl.ne, 0, qcs.QCS_FLAG_FP64_ALU, use_cache=args.tune_cache))
        s = qcs.Snapshots(ctx, torch.from_numpy(d["Q"]).to(dev), torch.from_numpy(d["b"]).to(dev))
        walkers = torch.from_numpy(d["Phi"]).to(dev)
        K = rng.standard_normal((wl.n, wl.n)) + 1j * rng.standard_normal((wl.n, wl.n))
        K = 0.01 * (K - K.conj().T)
        w, v = np.linalg.eigh(-1j * K)
        Us.append(torch.from_numpy((v * np.exp(1j * w)) @ v.conj().T).to(dev))
        systems.append((wl, s, walkers))
        outs.append(torch.empty(wl.W, dtype=torch.complex128, device=dev))
    pairs_step = sum(wl.W * wl.P for wl, _, _ in systems)
    # algorithmic FP64 flops of one step: parity +1 pairs of every system times its per-pair count
    flops_step = sum(wl.W * int((s.parity() == 1).sum().item()) * qcs.flops_per_pair(wl.n, wl.ne)
                     for wl, s, _ in systems)
    arg = [(s, w) for _, s, w in systems]

    def step():
        for (wl, s, w), U in zip(systems, Us):
            w.copy_(torch.matmul(U, w))
        qcs.overlap_batched(ctx, arg, outs=outs)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(args.batch_steps):
            step()
    torch.cuda.synchronize()
    barrier()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.replay()
    e1.record(stream)
    barrier()
    t = e0.elapsed_time(e1) / 1e3
    t = max_over_ranks(t, ws)
    # the pair kernel's own time per step (one batched call outside the graph, timed on its
    # launch), and each system alone in the same kernel, for context
    ctx.profile(True)
    ctx.profile_read()
    qcs.overlap_batched(ctx, arg, outs=outs)
    torch.cuda.synchronize()
    kms, _ = ctx.profile_read()
    per_sys = []
    for (wl, s, w) in systems:
        qcs.overlap_batched(ctx, [(s, w)])
        torch.cuda.synchronize()
        ms1, _ = ctx.profile_read()
        per_sys.append({"n": wl.n, "pairs_per_s_alone": wl.W * wl.P / (ms1 * 1e-3), "kernel_ms_alone": ms1})
    # the same systems in split precision (QCS_TF32X3, one qcs_overlap per system; n = 20
    # and 24 on the 64-row tiles), against the FP64 batched results of the same walkers
    split_rows, split_ms = [], 0.0
    for (wl, s, w), o_ref in zip(systems, outs):
        qcs.overlap(ctx, s, w, precision=qcs.QCS_TF32X3)  # builds the snapshot slabs once
        torch.cuda.synchronize()
        ctx.profile_read()
        o_split, _ = qcs.overlap(ctx, s, w, precision=qcs.QCS_TF32X3)
        torch.cuda.synchronize()
        ms1, _ = ctx.profile_read()
        split_ms += ms1
        split_rows.append({"n": wl.n, "pairs_per_s": wl.W * wl.P / (ms1 * 1e-3), "kernel_ms": ms1,
                           "walker_rel_diff_vs_fp64_max": float(((o_split - o_ref).abs() / o_ref.abs()).max().item())})
    ctx.profile(False)
    assert ctx.sync_status() == 0
    kach = flops_step / (kms * 1e-3) / 1e12
    return {"metric": "walker x snapshot overlap pairs/s, batched active spaces under a CUDA graph",
            "value": ws * pairs_step * args.batch_steps / t, "unit": "pairs/s",
            "ms_per_step": 1e3 * t / args.batch_steps, "graph_steps": args.batch_steps,
            "config": {"systems": [{"n": wl.n, "ne": wl.ne, "walkers": wl.W, "snapshots": wl.P,
                                    "tuned": qcs.decode_config(tc)} for (wl, _, _), tc in zip(systems, tuned)],
                       "picked_by": "qcs_autotune (QCS_FLAG_FP64_ALU, staged search: node rounds, tile, warps per pair)",
                       "walker_scale": args.batch_walker_scale,
                       "pairs_per_step": pairs_step,
                       "step": "stand-in propagation (torch matmul) + one qcs_overlap_batched launch sequence"},
            "roofline": {"bound": "alu", "achieved": flops_step * args.batch_steps / t / 1e12, "peak": FP64_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": flops_step * args.batch_steps / t / 1e12 / FP64_PEAK_TFLOPS,
                         "kernel": "pair_overlap_kernel (batched)",
                         "timing": "whole graph step (propagation, walker prep, pair kernel, reductions)"},
            "pair_kernel": {"kernel_ms_per_step": kms, "share_of_graph_step": kms / (1e3 * t / args.batch_steps),
                            "roofline": {"bound": "alu", "achieved": kach, "peak": FP64_PEAK_TFLOPS,
                                         "unit": "TFLOP/s", "frac": kach / FP64_PEAK_TFLOPS,
                                         "timing": "one batched launch outside the graph, events on its stream",
                                         "traffic": (traffic_for("pair_overlap_kernel_batched", BATCH_WORKLOAD)
                                                     if args.batch_walker_scale == 1.0 else None)}},
            "systems_alone": per_sys,
            "split_precision": {"systems": split_rows, "pairs_per_s_all": pairs_step / (split_ms * 1e-3),
                                "timing": "split kernel per system, events on its stream (no graph)"},
            "gpu_launches_per_step": 5 + 1 + 5}


def run_precision(args, ctx, dev, barrier, ws):
    """Split-precision workload: n = 16, ne = 8, 2048 walkers x 50000 snapshots; one step =
    snapshot build + qcs_overlap with QCS_TF32X3 (congruence on tcgen05 tensor cores as
    three TF32 hi/lo passes, B^(s) in FP32, Pfaffians in FP64).  Errors are measured
    against the FP64 path on the first 64 walkers x 4000 snapshots."""
    import torch
    import torch.distributed as dist

    from paper_2506_22408_gb300 import qcs, synth

    wl = synth.PRECISION
    if args.prec_walkers:
        import dataclasses

        wl = dataclasses.replace(wl, name=f"n={wl.n} ne={wl.ne} {args.prec_walkers}x{wl.P} (reduced profiling case)",
                                 W=args.prec_walkers)
    d = wl.generate(seed=0)
    Q = torch.from_numpy(d["Q"]).to(dev)
    b = torch.from_numpy(d["b"]).to(dev)
    Phi = torch.from_numpy(d["Phi"]).to(dev)
    del d

    def step():
        snaps = qcs.Snapshots(ctx, Q, b)
        ov, _ = qcs.overlap(ctx, snaps, Phi, precision=qcs.QCS_TF32X3)
        return snaps, ov

    snaps, _ = step()
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    npar = int((snaps.parity() == 1).sum().item())
    del snaps
    steps = max(2, min(args.steps, 3))
    ctx.profile(True)
    ctx.profile_read()
    barrier()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        snaps, ov = step()
    e1.record(stream)
    barrier()
    ctx.profile(False)
    kms, kl = ctx.profile_read()
    t = e0.elapsed_time(e1) / 1e3
    t = max_over_ranks(t, ws)
    # error against the FP64 path on a subset
    Ws, Ps = 64, 4000
    sub = qcs.Snapshots(ctx, Q[:Ps].contiguous(), b[:Ps].contiguous())
    o64, p64 = qcs.overlap(ctx, sub, Phi[:Ws].contiguous(), per_pair=True)
    o32, p32 = qcs.overlap(ctx, sub, Phi[:Ws].contiguous(), per_pair=True, precision=qcs.QCS_TF32X3)
    torch.cuda.synchronize()
    mag = p64.abs().mean(dim=1, keepdim=True)
    rel_pair = ((p32 - p64).abs() / mag).flatten()
    rel_walker = ((o32 - o64).abs() / mag.flatten())
    n, ne = wl.n, wl.ne
    f_pf = qcs.flops_breakdown(n, ne)["pfaffian"]  # FP64 work that stays on the FP64 pipe
    avg = kms / max(kl, 1)
    ach = f_pf * npar * wl.W / (avg * 1e-3) / 1e12
    ngroups = (wl.W + 3) // 4
    tensor_flops = ngroups * ((npar + 3) // 4) * 3 * 2.0 * 128 * 128 * 32  # tiles of 4 walkers x 4 snapshots
    return {"metric": "walker x snapshot overlap pairs/s, split precision (3xTF32 congruence on tensor cores)",
            "value": ws * wl.W * wl.P * steps / t, "unit": "pairs/s", "ms_per_step": 1e3 * t / steps,
            "steps": steps, "dtype": "tf32x3 congruence / f32 B / f64 Pfaffian",
            "config": {"workload": wl.name + " (Haar Q, uniform b, seed 0)", "parity_plus_snapshots": npar},
            "error_vs_fp64": {"subset": f"{Ws} walkers x {Ps} snapshots",
                              "pair_rel_max": float(rel_pair.max().item()),
                              "pair_rel_median": float(rel_pair.median().item()),
                              "walker_rel_max": float(rel_walker.max().item()),
                              "normalisation": "mean |o_p| of the walker on the FP64 path (per pair over s_p: cpu_baseline.parity.split_tf32x3)"},
            "roofline": {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": ach / FP64_PEAK_TFLOPS, "kernel": "split_pair_kernel", "kernel_ms": avg,
                         "flops_counted": "FP64 Pfaffian work only (congruence on tensor cores)",
                         "tensor_tflops_executed": tensor_flops / (avg * 1e-3) / 1e12,
                         "traffic": traffic_for("split_pair_kernel", wl.name)}}


def run_dft_plan(args, ctx, wl, Qd, bd, Pd, flush, barrier, ws, npar, steps=3):
    """Paper-shaped overlaps with the inverse-DFT node plan (n-ne+1 roots of unity,
    floor/2+1 evaluated) instead of the default Gauss plan: same estimator, more
    Pfaffians per pair.  Reported beside the headline for comparison."""
    import torch

    from paper_2506_22408_gb300 import qcs

    flags = qcs.QCS_FLAG_DFT_NODES
    ctx.autotune(wl.n, wl.ne, 0, flags, use_cache=args.tune_cache)
    stream = torch.cuda.current_stream()

    def step():
        snaps = qcs.Snapshots(ctx, Qd, bd)
        qcs.overlap(ctx, snaps, Pd, flags=flags)
        return snaps

    for _ in range(2):
        step()
    barrier()
    ctx.profile(True)
    ctx.profile_read()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    barrier()
    ctx.profile(False)
    kms, kl = ctx.profile_read()
    assert ctx.sync_status() == 0
    t = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / 1e3, ws)
    fpp = qcs.tc_work_per_pair(wl.n, wl.ne, 0, flags)["fp64"]
    avg = kms / max(kl, 1)
    ach = fpp * npar * wl.W / (avg * 1e-3) / 1e12
    return {"metric": "walker x snapshot overlap pairs/s, roots-of-unity node plan", "value": ws * wl.W * wl.P * steps / t,
            "unit": "pairs/s", "steps": steps, "ms_per_step": 1e3 * t / steps,
            "nodes": f"{len(qcs.node_plan(wl.n, wl.ne, 0, flags)[0])} of {wl.n - wl.ne + 1} roots of unity",
            "roofline": {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": ach / FP64_PEAK_TFLOPS, "kernel": "tc_pair_kernel", "kernel_ms": avg,
                         "flops_per_launch": fpp * npar * wl.W}}


def run_alu_path(args, ctx, wl, Qd, bd, Pd, flush, barrier, ws, npar, steps=3):
    """The same workload (1024 x 20000, n=16, ne=8, Gauss plan) with the congruence on
    the FP64 ALU (QCS_FLAG_FP64_ALU), the plain GPU path the tensor-core congruence is
    measured against."""
    import torch

    from paper_2506_22408_gb300 import qcs

    flags = qcs.QCS_FLAG_FP64_ALU
    tuned = ctx.autotune(wl.n, wl.ne, 0, flags, use_cache=args.tune_cache)
    stream = torch.cuda.current_stream()

    def step():
        snaps = qcs.Snapshots(ctx, Qd, bd)
        qcs.overlap(ctx, snaps, Pd, flags=flags)
        return snaps

    for _ in range(2):
        step()
    barrier()
    ctx.profile(True)
    ctx.profile_read()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    barrier()
    ctx.profile(False)
    kms, kl = ctx.profile_read()
    assert ctx.sync_status() == 0
    t = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / 1e3, ws)
    fpp = qcs.flops_per_pair(wl.n, wl.ne, 0, flags)
    avg = kms / max(kl, 1)
    ach = fpp * npar * wl.W / (avg * 1e-3) / 1e12
    return {"metric": "walker x snapshot overlap pairs/s, congruence on the FP64 ALU", "value": ws * wl.W * wl.P * steps / t,
            "unit": "pairs/s", "steps": steps, "ms_per_step": 1e3 * t / steps,
            "nontrivial_pairs_per_s": ws * wl.W * npar * steps / t,
            "kernel_config": {**qcs.decode_config(tuned), "picked_by": "qcs_autotune (QCS_FLAG_FP64_ALU)"},
            "roofline": {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": ach / FP64_PEAK_TFLOPS, "kernel": "pair_overlap_kernel", "kernel_ms": avg,
                         "flops_per_launch": fpp * npar * wl.W,
                         "traffic": traffic_for("pair_overlap_kernel", wl.name)}}


def run_variants(args, ctx, dev, flush, barrier, ws, steps=3):
    """The paper-shaped size (1024 x 20000, n=16, ne=8) with other snapshot
    ensembles: b uniform over the parity-consistent strings (every pair
    non-trivial), and signed-permutation snapshots (the paper's ensemble), with
    uniform and with parity-consistent b; the default (tensor-core) path."""
    import dataclasses

    import torch

    from paper_2506_22408_gb300 import qcs, synth

    stream = torch.cuda.current_stream()
    out = {}
    for key, ens, bits in (("haar_parity_b", "haar", "parity"), ("signed_perm_uniform_b", "signed_perm", "uniform"),
                           ("signed_perm_parity_b", "signed_perm", "parity")):
        wl = dataclasses.replace(synth.PAPER_SHAPED, name=f"paper-shaped {ens} Q, {bits} b", ensemble=ens, bits=bits)
        if args.walkers or args.snapshots:
            wl = dataclasses.replace(wl, W=args.walkers or wl.W, P=args.snapshots or wl.P)
        d = wl.generate(seed=0)
        Qd, bd, Pd = (torch.from_numpy(d[k]).to(dev) for k in ("Q", "b", "Phi"))

        def step():
            snaps = qcs.Snapshots(ctx, Qd, bd)
            qcs.overlap(ctx, snaps, Pd)
            return snaps

        for _ in range(2):
            snaps = step()
        barrier()
        npar = int((snaps.parity() == 1).sum().item())
        nsp = snaps.signed_perm_count()
        del snaps
        ctx.profile(True)
        ctx.profile_read()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        barrier()
        ctx.profile(False)
        kms, kl = ctx.profile_read()
        assert ctx.sync_status() == 0
        t = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / 1e3, ws)
        fpp = qcs.tc_work_per_pair(wl.n, wl.ne)["fp64"]  # the default path at n = 16: tensor-core congruence
        avg = kms / max(kl, 1)
        ach = fpp * npar * wl.W / (avg * 1e-3) / 1e12
        out[key] = {"value": ws * wl.W * wl.P * steps / t, "unit": "pairs/s",
                    "nontrivial_pairs_per_s": ws * wl.W * npar * steps / t, "steps": steps,
                    "parity_plus_snapshots": npar, "signed_perm_snapshots": nsp,
                    "roofline": {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                                 "frac": ach / FP64_PEAK_TFLOPS, "kernel": "tc_pair_kernel", "kernel_ms": avg,
                                 "flops_per_pair": fpp}}
        del Qd, bd, Pd
    return out


def run_rdm(args, ctx, dev, flush, barrier, ws, steps=3):
    """Shadow RDM estimates (Supplementary "Reduced Density Matrices") from the
    paper's shadow count: n=16, 60000 Haar snapshots, uniform b; one step builds the
    snapshot set and runs qcs_shadow_rdm with the four-Majorana estimates."""
    import torch

    from paper_2506_22408_gb300 import qcs, synth

    n, P = 16, args.rdm_snapshots
    rng = np.random.default_rng(0)
    Qd = torch.from_numpy(synth.haar_orthogonal(rng, 2 * n, P)).to(dev)
    bd = torch.from_numpy(synth.uniform_bits(rng, n, P)).to(dev)
    stream = torch.cuda.current_stream()

    def step():
        snaps = qcs.Snapshots(ctx, Qd, bd)
        return qcs.shadow_rdm(ctx, snaps, deg4=True)

    for _ in range(2):
        step()
    barrier()
    ctx.profile(True)
    ctx.profile_read()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        out = step()
        ev[i][1].record(stream)
    barrier()
    ctx.profile(False)
    kms, kl = ctx.profile_read()
    assert ctx.sync_status() == 0
    t = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / 1e3, ws)
    avg = kms / max(kl, 1)
    fl = qcs.shadow_rdm_flops(n, P)
    ach = fl / (avg * 1e-3) / 1e12
    return {"metric": "snapshots/s, shadow estimates of the 1-RDM, particle number and all four-Majorana correlators",
            "value": ws * P * steps / t, "unit": "snapshots/s", "steps": steps, "ms_per_step": 1e3 * t / steps,
            "config": {"workload": f"shadow RDM n={n} {P} snapshots (Haar Q, uniform b, seed 0)"},
            "particle_number": float(out["npart"].item()),
            "roofline": {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": ach / FP64_PEAK_TFLOPS, "kernel": "rdm_syrk_kernel", "kernel_ms": avg,
                         "flops_per_launch": fl,
                         "traffic": traffic_for("rdm_syrk_kernel", f"shadow RDM n={n} {P} snapshots")}}


def run_vce(args, ctx, dev, flush, barrier, ws, steps=3):
    """Virtual-correlation-energy path: full-space unrestricted walkers (200 orbitals
    and 20 + 4 electrons per spin, 20 core orbitals) mapped by qcs_vce_transform onto
    the paper-shaped active space (8 orbitals and 4 electrons per spin: n=16, ne=8),
    then the shadow overlap with 20000 snapshots; one step = both transforms and the
    overlap.  The transform alone is also timed."""
    import torch

    from paper_2506_22408_gb300 import qcs, synth

    NB, nc, na, nea, W, P = 200, 20, 8, 4, 1024, 20000
    rng = np.random.default_rng(0)
    Pa = torch.from_numpy(rng.standard_normal((W, NB, nc + nea)) + 1j * rng.standard_normal((W, NB, nc + nea))).to(dev)
    Pb = torch.from_numpy(rng.standard_normal((W, NB, nc + nea)) + 1j * rng.standard_normal((W, NB, nc + nea))).to(dev)
    Qd = torch.from_numpy(synth.haar_orthogonal(rng, 4 * na, P)).to(dev)
    bd = torch.from_numpy(synth.uniform_bits(rng, 2 * na, P)).to(dev)
    act = torch.zeros((W, 2 * na, 2 * nea), dtype=torch.complex128, device=dev)
    stream = torch.cuda.current_stream()

    def transform():
        _, fa = qcs.vce_transform(ctx, Pa, nc, na, nea, act=act, row0=0, col0=0)
        _, fb = qcs.vce_transform(ctx, Pb, nc, na, nea, act=act, row0=na, col0=nea)
        return fa, fb

    def step():
        fa, fb = transform()
        snaps = qcs.Snapshots(ctx, Qd, bd)
        ov, _ = qcs.overlap(ctx, snaps, act)
        return ov * fa * fb

    for _ in range(2):
        step()
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    barrier()
    assert ctx.sync_status() == 0
    t = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / 1e3, ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    e0.record(stream)
    for _ in range(reps):
        transform()
    e1.record(stream)
    barrier()
    tt = e0.elapsed_time(e1) / 1e3 / reps
    return {"metric": "full-space walker x snapshot overlap pairs/s through the VCE transform", "unit": "pairs/s",
            "value": ws * W * P * steps / t, "steps": steps, "ms_per_step": 1e3 * t / steps,
            "transform_walkers_per_s": ws * 2 * W / tt,
            "config": {"workload": f"VCE NB={NB} per spin, {nc} core, active {na} orbitals / {nea} electrons "
                                   f"per spin (n=16, ne=8), {W} walkers x {P} snapshots"}}


def run_energy(args, ctx, dev, flush, barrier, ws, steps=2):
    """Local-energy terms (Eqs. energy_tb_diff, Pfaffian_2nd_der): n=16, ne=8, 64 walkers
    x 1000 snapshots, 64 Cholesky vectors and a one-body operator; one step = snapshot
    build + qcs_local_energy."""
    import torch

    from paper_2506_22408_gb300 import qcs, synth

    n, ne, W, P, nchol = 16, 8, args.energy_walkers, 1000, 64
    rng = np.random.default_rng(0)
    Qd = torch.from_numpy(synth.haar_orthogonal(rng, 2 * n, P)).to(dev)
    bd = torch.from_numpy(synth.uniform_bits(rng, n, P)).to(dev)
    Pd = torch.from_numpy(synth.walkers(rng, n, ne, W)).to(dev)
    Ld = torch.from_numpy(synth.cholesky_vectors(rng, n, nchol).astype(complex)).to(dev)
    hd = torch.from_numpy(synth.cholesky_vectors(rng, n, 1)[0].astype(complex)).to(dev)
    stream = torch.cuda.current_stream()

    def step():
        snaps = qcs.Snapshots(ctx, Qd, bd)
        qcs.local_energy(ctx, snaps, Pd, Ld, hd)
        return snaps

    snaps = step()
    barrier()
    npar = int((snaps.parity() == 1).sum().item())
    ctx.profile(True)
    ctx.profile_read()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    barrier()
    ctx.profile(False)
    kms, kl = ctx.profile_read()
    assert ctx.sync_status() == 0
    t = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / 1e3, ws)
    fpp = qcs.local_energy_flops_per_pair(n, ne, nchol, True)
    avg = kms / max(kl, 1)
    ach = fpp * npar * W / (avg * 1e-3) / 1e12
    return {"metric": "walker x snapshot pairs/s, local-energy terms (overlap, one-body and two-body)",
            "value": ws * W * P * steps / t, "unit": "pairs/s", "steps": steps, "ms_per_step": 1e3 * t / steps,
            "config": {"workload": f"local energy n={n} ne={ne} {W}x{P} nchol={nchol} (Haar Q, uniform b, seed 0)",
                       "parity_plus_snapshots": npar},
            "roofline": {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": ach / FP64_PEAK_TFLOPS, "kernel": "energy_pair_kernel", "kernel_ms": avg,
                         "flops_per_launch": fpp * npar * W,
                         "traffic": traffic_for("energy_pair_kernel", f"local energy n={n} ne={ne} {W}x{P} nchol={nchol}")}}


def cpu_baseline(wl, data, gpu_overlap, gpu_sample, target_s=10.0):
    """The CPU oracle, as it stands, on a bounded sample of the workload; the same oracle
    results also give the parity of the GPU path at the benchmark's size: every pair of
    the sample (|o_gpu - o_oracle| / s_p, s_p the magnitude of the pair's terms before
    they cancel, and exact zeros for parity -1), the sample's walker means, and three
    whole walkers over all snapshots against the overlaps of the timed steps (relative
    to |O|).  gpu_sample(Wc, Pc) returns the GPU's walker and per-pair outputs on the
    sample, the parity flags and a dict of per-pair outputs of other paths (checked pair
    by pair against s_p as well); gpu_overlap holds the timed steps' walker overlaps."""
    import numpy as np

    import oracle.oracle as orc

    cores = orc.max_threads()
    Wc = min(64, wl.W)
    Pc = min(wl.P, 200)
    t0 = time.perf_counter()
    orc.overlap(data["Phi"][:Wc], data["Q"][:Pc], data["b"][:Pc], threads=cores)
    dt = time.perf_counter() - t0
    # grow the sample to about target_s seconds of CPU work
    Pc2 = int(min(wl.P, max(Pc, Pc * target_s / max(dt, 1e-3))))
    t0 = time.perf_counter()
    oo, opp, sc, used = orc.overlap(data["Phi"][:Wc], data["Q"][:Pc2], data["b"][:Pc2], threads=cores, per_pair=True)
    dt = time.perf_counter() - t0
    # the same oracle on one host thread, on a smaller sample (about 2 s)
    P1 = max(1, min(Pc2, int(Pc2 * 2.0 / max(dt * used, 1e-3))))
    t0 = time.perf_counter()
    orc.overlap(data["Phi"][:Wc], data["Q"][:P1], data["b"][:P1], threads=1)
    dt1 = time.perf_counter() - t0
    # parity: the sample pair by pair, its walker means, and three whole walkers
    gov, gpp, gpar, other_paths = gpu_sample(Wc, Pc2)
    ok = gpar == 1
    pair_err = np.abs(gpp[:, ok] - opp[:, ok]) / sc[:, ok]
    sample_rel = np.abs(gov - oo) / np.abs(oo)
    sel = np.array([0, wl.W // 2, wl.W - 1])
    fo, _, fsc, _ = orc.overlap(data["Phi"][sel], data["Q"], data["b"], threads=cores, per_pair=True)
    full_rel = np.abs(gpu_overlap[sel] - fo) / np.abs(fo)
    orc.overlap(data["Phi"][:1], data["Q"][:1], data["b"][:1], threads=cores)  # restore the thread count
    parity = {"pairs": int(ok.sum()) * Wc, "pair_err_over_scale_max": float(pair_err.max()),
              "pair_err_over_scale_median": float(np.median(pair_err)),
              "parity_minus_pairs_exactly_zero": bool(np.all(gpp[:, ~ok] == 0)),
              "sample_walkers": Wc, "sample_walker_rel_err_max": float(sample_rel.max()),
              "sample_walker_rel_err_median": float(np.median(sample_rel)),
              "full_walkers": sel.tolist(), "full_walker_rel_err": [float(x) for x in full_rel],
              "full_walker_cancellation": [float(x) for x in fsc.mean(axis=1) / np.abs(fo)],
              "tolerance": "pairs 1e-10 s_p, walkers 1e-10 relative",
              "within_tolerance": bool(pair_err.max() <= 1e-10 and sample_rel.max() <= 1e-10
                                       and full_rel.max() <= 1e-10 and np.all(gpp[:, ~ok] == 0))}
    # the same sample through the FP64 ALU congruence and the split precision (bound 2e-5 s_p)
    for name, opp_path in other_paths.items():
        e = np.abs(opp_path[:, ok] - opp[:, ok]) / sc[:, ok]
        parity[name] = {"pair_err_over_scale_max": float(e.max()),
                        "pair_err_over_scale_median": float(np.median(e)),
                        "parity_minus_pairs_exactly_zero": bool(np.all(opp_path[:, ~ok] == 0)),
                        "bound": 2e-5 if name.startswith("split") else 1e-10}
    return {"value": Wc * Pc2 / dt, "unit": "pairs/s", "cores": int(used), "kind": "oracle",
            "sample": f"{Wc} walkers x {Pc2} snapshots of the same workload (first rows), "
                      f"{dt:.1f} s, FP64, 2n+1 roots-of-unity nodes, OpenMP over pairs",
            "one_thread": {"value": Wc * P1 / dt1, "unit": "pairs/s",
                           "sample": f"{Wc} walkers x {P1} snapshots, {dt1:.1f} s"},
            "cpu_model": cpu_model(), "parity": parity}


def cpu_model() -> str:
    """The host CPU's model name (Linux), else the platform's processor string."""
    import platform

    part = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware") and ":" in line:
                    return line.split(":", 1)[1].strip()
                if key == "cpu part" and part is None:  # Arm cores list an implementer part number
                    part = line.split(":", 1)[1].strip()
    except OSError:
        pass
    base = platform.processor() or platform.machine()
    return f"{base}, CPU part {part}" if part else base


def run_reference(args, wl):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle.oracle as orc

    Wc = min(64, wl.W)
    data = wl.generate(seed=0, W=Wc, P=min(wl.P, 4000))
    cores = orc.max_threads()
    # size each step at a few seconds of CPU work
    t0 = time.perf_counter()
    P0 = min(100, wl.P)
    orc.overlap(data["Phi"][:Wc], data["Q"][:P0], data["b"][:P0], threads=cores)
    per_pair = (time.perf_counter() - t0) / (Wc * P0)
    Pc = int(min(4000, wl.P, max(100, 4.0 / max(per_pair * Wc, 1e-9))))
    for _ in range(args.warmup):
        orc.overlap(data["Phi"][:Wc], data["Q"][:Pc], data["b"][:Pc], threads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        orc.overlap(data["Phi"][:Wc], data["Q"][:Pc], data["b"][:Pc], threads=cores)
        times.append(time.perf_counter() - t0)
    T = sum(times)
    val = Wc * Pc * args.steps / T
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "pairs/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "n": wl.n, "ne": wl.ne, "walkers": wl.W, "snapshots": wl.P,
                       "sample_per_step": f"{Wc} walkers x {Pc} snapshots"},
            "cpu_baseline": {"value": val, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                             "sample": f"{Wc} walkers x {Pc} snapshots per step"},
            "e2e": {"value": val, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-grad", action="store_true", help="skip the differentiation workload")
    ap.add_argument("--grad-walkers", type=int, default=0, help="override the differentiation walkers (profiling)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batching workload")
    ap.add_argument("--no-precision", action="store_true", help="skip the split-precision workload")
    ap.add_argument("--no-dft-plan", action="store_true", help="skip the roots-of-unity node-plan comparison")
    ap.add_argument("--no-alu-path", action="store_true", help="skip the FP64 ALU congruence comparison")
    ap.add_argument("--tune-cache", action="store_true",
                    help="take the autotuner's choices from its cache file when present (default: tune in this run)")
    ap.add_argument("--no-rdm", action="store_true", help="skip the shadow RDM workload")
    ap.add_argument("--no-vce", action="store_true", help="skip the virtual-correlation-energy workload")
    ap.add_argument("--no-energy", action="store_true", help="skip the local-energy workload")
    ap.add_argument("--energy-walkers", type=int, default=64, help="walkers of the local-energy workload")
    ap.add_argument("--rdm-snapshots", type=int, default=60000, help="snapshots of the shadow RDM workload")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the parity-consistent and signed-permutation snapshot ensembles")
    ap.add_argument("--prec-walkers", type=int, default=0, help="override the split-precision walkers (profiling)")
    ap.add_argument("--batch-steps", type=int, default=50, help="AFQMC steps captured in the batching graph")
    ap.add_argument("--batch-walker-scale", type=float, default=1.0,
                    help="scale of the batching walker counts (1.0: 1024/512/256/128/64 walkers)")
    ap.add_argument("--grad-snapshots", type=int, default=0, help="override the differentiation snapshots")
    ap.add_argument("--walkers", type=int, default=0, help="override the walker count (profiling cases)")
    ap.add_argument("--snapshots", type=int, default=0, help="override the snapshot count (profiling cases)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    from paper_2506_22408_gb300 import synth

    wl = synth.PAPER_SHAPED
    if args.walkers or args.snapshots:
        import dataclasses

        W = args.walkers or wl.W
        P = args.snapshots or wl.P
        wl = dataclasses.replace(wl, name=f"n={wl.n} ne={wl.ne} {W}x{P} (reduced profiling case)", W=W, P=P)
    if args.impl == "reference":
        return run_reference(args, wl)

    import torch
    import torch.distributed as dist

    from paper_2506_22408_gb300 import qcs

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("gloo", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    data = wl.generate(seed=0)
    ctx = qcs.Context(local)
    tuned = ctx.autotune(wl.n, wl.ne, use_cache=args.tune_cache)  # kernel configuration for this GPU
    Qd = torch.from_numpy(data["Q"]).to(dev)
    bd = torch.from_numpy(data["b"]).to(dev)
    Pd = torch.from_numpy(data["Phi"]).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(Q, b, Phi):
        snaps = qcs.Snapshots(ctx, Q, b)
        ov, _ = qcs.overlap(ctx, snaps, Phi)
        return snaps, ov

    for _ in range(args.warmup):
        snaps, ov = step(Qd, bd, Pd)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    npar = int((snaps.parity() == 1).sum().item())
    del snaps

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---------------- device-resident timed region
    ctx.profile(True)
    ctx.profile_read()
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with Clocks(local) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))  # L2 flush between steps, outside the timed events
            ev[i][0].record(stream)
            snaps, ov = step(Qd, bd, Pd)
            ev[i][1].record(stream)
        barrier()
    ctx.profile(False)
    kern_ms, kern_launches = ctx.profile_read()
    ov_timed = ov.cpu().numpy()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_total = sum(step_ms) / 1e3
    t_total = max_over_ranks(t_total, ws)
    pairs = wl.W * wl.P
    value = ws * pairs * args.steps / t_total
    del snaps

    # ---------------- the same workload with the roots-of-unity node plan
    dft = None
    if not args.no_dft_plan:
        dft = run_dft_plan(args, ctx, wl, Qd, bd, Pd, flush, barrier, ws, npar)

    # ---------------- other snapshot ensembles at the same size
    variants = None
    if not args.no_variants:
        variants = run_variants(args, ctx, dev, flush, barrier, ws)

    # ---------------- shadow RDM estimates (walker-independent)
    rdm = None
    if not args.no_rdm:
        rdm = run_rdm(args, ctx, dev, flush, barrier, ws)

    # ---------------- virtual-correlation-energy path
    vce = None
    if not args.no_vce:
        vce = run_vce(args, ctx, dev, flush, barrier, ws)

    # ---------------- local-energy terms
    energy = None
    if not args.no_energy:
        energy = run_energy(args, ctx, dev, flush, barrier, ws)

    # ---------------- end to end through the C ABI from pinned host buffers
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, data, dev, step, barrier, ws, wl)
    alu = None
    if not args.no_alu_path:
        alu = run_alu_path(args, ctx, wl, Qd, bd, Pd, flush, barrier, ws, npar)
    grad = None
    if not args.no_grad:
        grad = run_grad(args, ctx, dev, barrier, ws)
    batch = None
    if not args.no_batch:
        batch = run_batch(args, ctx, dev, barrier, ws)
    precision = None
    if not args.no_precision:
        precision = run_precision(args, ctx, dev, barrier, ws)

    # ---------------- roofline of the dominant kernel (tensor-core congruence, n = 16)
    work = qcs.tc_work_per_pair(wl.n, wl.ne)
    fpp, tpp = work["fp64"], work["tensor"]
    alu_fpp = qcs.flops_per_pair(wl.n, wl.ne, 0, qcs.QCS_FLAG_FP64_ALU)
    avg_ms = kern_ms / max(kern_launches, 1)
    pairs_launch = npar * wl.W
    achieved = fpp * pairs_launch / (avg_ms * 1e-3) / 1e12
    tensor_ach = tpp * pairs_launch / (avg_ms * 1e-3) / 1e12
    peaks = measured_peaks()
    bf16 = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
    roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic_for("tc_pair_kernel", wl.name),
            "kernel": "tc_pair_kernel", "kernel_ms": avg_ms, "flops_per_launch": fpp * pairs_launch,
            "fp64_flops_per_pair": fpp,
            "peak_source": "FP64 ALU: 152 SM x 4 flop/clk x 2.07 GHz (derived from unit counts and the maximum "
                           "clock; MEASURED_PEAKS.json carries no FP64 figure)",
            "tensor": {"achieved": tensor_ach, "peak": bf16, "unit": "TFLOP/s",
                       "frac": tensor_ach / bf16 if bf16 else None, "bf16_flops_per_pair": tpp,
                       "peak_source": f"bf16_tflops_sustained ({peaks['source']}; cuBLAS bf16 timed inside a long loop)"},
            "fp64_alu_equivalent": {"flops_per_pair": alu_fpp,
                                    "tflops": alu_fpp * pairs_launch / (avg_ms * 1e-3) / 1e12,
                                    "note": "FP64 work the ALU congruence executes for the same result"}}

    line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name + " (Haar Q, uniform b, seed 0)", "n": wl.n, "ne": wl.ne,
                       "walkers": wl.W, "snapshots": wl.P, "parity_plus_snapshots": npar,
                       "nodes": f"Gauss plan: {len(qcs.node_plan(wl.n, wl.ne)[0])} Pfaffians per parity +1 pair",
                       "kernel_config": {**qcs.decode_config(tuned), "picked_by": "qcs_autotune"},
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "l2": "snapshot set (164 MB) larger than L2, and L2 flushed between timed steps"},
            "nontrivial_pairs_per_s": ws * npar * wl.W * args.steps / t_total,
            "e2e": e2e,
            "roofline": roof,
            "clocks": clk.summary(),
            "fp64_alu_congruence": alu,
            "grad": grad,
            "batch": batch,
            "precision": precision,
            "roots_of_unity_plan": dft,
            "ensembles": variants,
            "rdm": rdm,
            "vce": vce,
            "local_energy": energy,
            # per step: snapshot build (prepare, compaction, tensor-core records) and the
            # overlap (walker prep, walker slices, pair kernel, reduction)
            "gpu_launches": args.steps * 7}
    if rank == 0 and not args.no_cpu_baseline:
        def gpu_sample(Wc, Pc):
            s2 = qcs.Snapshots(ctx, Qd[:Pc].contiguous(), bd[:Pc].contiguous())
            o2, pp2 = qcs.overlap(ctx, s2, Pd[:Wc].contiguous(), per_pair=True)
            others = {}
            if wl.n == 16:  # the other two congruence paths on the same sample
                others["fp64_alu"] = qcs.overlap(ctx, s2, Pd[:Wc].contiguous(), per_pair=True,
                                                 flags=qcs.QCS_FLAG_FP64_ALU)[1]
                others["split_tf32x3"] = qcs.overlap(ctx, s2, Pd[:Wc].contiguous(), per_pair=True,
                                                     precision=qcs.QCS_TF32X3)[1]
            torch.cuda.synchronize()
            return (o2.cpu().numpy(), pp2.cpu().numpy(), s2.parity().cpu().numpy(),
                    {k: v.cpu().numpy() for k, v in others.items()})

        line["cpu_baseline"] = cpu_baseline(wl, data, ov_timed, gpu_sample)
    add_dfma_context(line, ctx.fp64_fma_rate())
    if ws > 1:
        dist.barrier()
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
