"""Benchmark of the Hamiltonian build (and Davidson) on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--config c3] [--precision mixed|fp64] [--fp64-steps 3]
                    [--davidson-k 20] [--davidson-config c2]

One step is one mixed-precision build of every class of the close-coupling
Hamiltonian (hb_build_blocks) for the precision workload (40 target + 400
continuum orbitals, N = 14 + 1 electrons, 20000 target determinants, 50 target
states, 30000 L2 functions, dimension 50000), with the integrals already
resident on the device.  The metric is H elements per second: dim(dim+1)/2
lower-triangle positions per build (the positions the paper's whole-matrix
timings cover).  The plain FP64 GPU build of the same instance is timed after
the steps ("fp64", "speedup_vs_fp64").  Davidson (lowest 20 eigenpairs of the
medium workload, dimension 8000, to a residual of 1e-8) is timed after that,
on the GPU and with the CPU baseline (numpy block Davidson), under "davidson";
the lowest 200 eigenpairs of the 60000-dimensional workload under
"davidson_c5"; the build and Davidson of the L2-heavy shape of the paper's
H3PO4 run (dimension 122815, 122103 L2 functions) under "l2_heavy"; the
16-Hamiltonian batched build under "batched".

Prints one JSON line (rank 0).  Under torchrun every rank builds its own
replica (independent problem, no data-path collective) and the time is the
maximum over ranks.  With --sharded the ranks also build one matrix together
(contraction shares, an NCCL all-reduce of the partial coefficient rows,
expansion shares) and the line gains a "sharded" key (strong scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CONFIG_TEXT = {
    "c1": "c1_tiny: 10 target + 20 continuum orbitals, N=6+1, 40 target dets, 3 states, 50 L2, dim 110",
    "c2": "c2_medium: 30 target + 150 continuum orbitals, N=10+1, 2000 target dets, 20 states, 5000 L2, dim 8000",
    "c3": "c3_precision: 40 target + 400 continuum orbitals, N=14+1, 20000 target dets, 50 states, 30000 L2, "
          "dim 50000",
}


def positions(dim):
    return dim * (dim + 1) / 2


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[0])); mx.append(float(f[1]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def overrides(args):
    """Integer workload sizes given with --set KEY=INT."""
    out = {}
    for kv in args.set:
        k, v = kv.split("=", 1)
        out[k.strip()] = int(v)
    return out


def workload_text(args):
    text = CONFIG_TEXT.get(args.config, args.config)
    if args.set:
        text += " with " + ", ".join(args.set)
    return text


def pinned_problem(P):
    """A copy of the problem whose arrays live in page-locked host memory."""
    import dataclasses
    import torch

    def pin(a):
        return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()

    groups = [dataclasses.replace(g, dets=pin(g.dets), ci=pin(g.ci)) for g in P.groups]
    return dataclasses.replace(P, h=pin(P.h), eri_tttt=pin(P.eri_tttt), eri_tttc=pin(P.eri_tttc),
                               eri_ttcc=pin(P.eri_ttcc), eri_tctc=pin(P.eri_tctc), l2_dets=pin(P.l2_dets),
                               groups=groups)


def profiled_traffic(kernel, source, config):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on this workload and the kernel source has not changed since the
    counters were taken (else None)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(kernel)
        with open(os.path.join(ROOT, source), "rb") as f:
            sha = hashlib.sha1(f.read()).hexdigest()
    except (OSError, ValueError):
        return None
    if not rec or rec.get("source_sha1") != sha or rec.get("config") != config:
        return None
    return rec.get("dram_bytes_per_launch")


def class4_roofline(n_l2, contracted_dim, kernel_ms, peaks):
    """HBM roofline of the class-4 kernels (Eq. 5) from the floor of their
    algorithmic bytes: the Hlc block, n_l2 x contracted dim in FP64, written
    once.  The integral and CI rows they gather come on top of that floor, so
    the fraction is an upper bound on how much of HBM the work needs."""
    if not kernel_ms or kernel_ms <= 0 or n_l2 <= 0 or contracted_dim <= 0:
        return None
    nbytes = 8.0 * n_l2 * contracted_dim
    hbm = peaks.get("hbm_gbs")
    achieved = nbytes / (kernel_ms / 1e3) / 1e9
    return {"bound": "hbm", "unit": "GB/s", "kernel": "class 4 (Eq. 5): class4_tc_kernel / class4_df_kernel",
            "bytes_per_launch": nbytes,
            "bytes_definition": "the Hlc block written once (n_l2 x contracted dim x 8 B); gathered integral and "
                                "CI rows not counted",
            "kernel_ms": kernel_ms, "achieved": achieved, "peak": hbm,
            "peak_source": "measured HBM copy (of measured)",
            "frac": achieved / hbm if hbm else None}


def fp64_alu_peak_tflops():
    # GB300 nominal FP64 1.25 TFLOP/s = 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz
    return 152 * 2 * 2 * 2.07e9 / 1e12


def fp64_projection_rate(dst):
    """Davidson's FP64 projections and basis combinations (Gram sums, norms,
    project-outs, combines) against the FP64 pipe: their flops over the time the
    solver spends in them (which includes the host waits on those results)."""
    ms = dst.ms_gram + dst.ms_combine
    tf = dst.proj_gflop * 1e9 / (ms / 1e3) / 1e12 if ms > 0 else None
    return {"gflop": dst.proj_gflop, "ms": ms, "achieved_tflops": tf, "peak_tflops": fp64_alu_peak_tflops(),
            "peak_source": "derived FP64 peak: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz",
            "frac": tf / fp64_alu_peak_tflops() if tf else None}


def cpu_baseline(problem, budget_s=20.0):
    """Time the oracle (as it stands) on this host's cores on the same workload,
    or on a bounded sample of it.  Every group-pair contraction (Eq. 8) runs in
    full; then each of the three expansion stages (continuum rows of Eq. 7,
    class-4 rows of Eq. 5, L2 rows) runs on leading rows until its share of the
    budget is spent.  A stage that did not finish is extrapolated to all of its
    rows at the rate measured, so the value is the whole workload's positions
    over the whole workload's estimated oracle time (contraction included)."""
    from oracle import coracle
    o = coracle.Oracle(problem)
    gs = problem.groups
    share = budget_s / 3.0
    t_contract = t_cc = 0.0
    cc_done = cc_all = 0.0
    npairs = len(gs) * (len(gs) + 1) // 2
    for g in range(len(gs)):
        for gp in range(g + 1):
            t0 = time.perf_counter()
            cc = o.contract(g, gp, cond=False)
            t_contract += time.perf_counter() - t0
            cn = gs[g].cont_count
            per_row = gs[g].ci.shape[1] * gs[gp].ci.shape[1] * gs[gp].cont_count
            cc_all += cn * per_row
            step = max(1, cn // 16)
            for jj0 in range(0, cn, step):
                if t_cc > share * (g * (g + 1) // 2 + gp + 1) / npairs:
                    break
                jj1 = min(cn, jj0 + step)
                t0 = time.perf_counter()
                cc.expand_rows(jj0, jj1)
                t_cc += time.perf_counter() - t0
                cc_done += (jj1 - jj0) * per_row
            del cc
    stages = [("contraction", t_contract, 1.0)]
    stages.append(("expansion", t_cc, cc_done / max(cc_all, 1.0)))
    nl = problem.n_l2
    for name, fn in (("class 4", o.class4_rows), ("L2", o.l2_rows)):
        if not nl:
            break
        t, done, step = 0.0, 0, 64
        while done < nl and t < share:
            n = min(step, nl - done)
            t0 = time.perf_counter()
            fn(done, done + n)
            t += time.perf_counter() - t0
            done += n
            step *= 2
        stages.append((name, t, done / nl))
    est = stages[0][1] + sum(t / f for _, t, f in stages[1:] if f > 0)
    measured = sum(t for _, t, _ in stages)
    full = all(f >= 1.0 for _, _, f in stages)
    detail = ", ".join(f"{n} {100 * f:.1f} % in {t:.2f} s" for n, t, f in stages[1:])
    what = "whole workload: every block once" if full else \
        f"bounded sample of {problem.name}: every contraction ({t_contract:.2f} s), then {detail}; unfinished " \
        f"stages extrapolated at their measured rate to {est:.1f} s for the whole workload"
    return {"value": positions(problem.dim) / est, "unit": "H elements/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{what} ({measured:.1f} s measured)"}


def cpu_davidson(problem, k, tol=1e-8):
    """CPU baseline of the Davidson step: the oracle's plain numpy block
    Davidson (FP64, OpenBLAS on all host cores) on the oracle's dense matrix
    of the same instance; the dense build itself is not timed."""
    from oracle import coracle, eig
    H = coracle.Oracle(problem).dense()
    d = np.ascontiguousarray(np.diag(H))
    t0 = time.perf_counter()
    w, X, it = eig.davidson(lambda V: H @ V, d, k, tol=tol, max_iter=400)
    dt = time.perf_counter() - t0
    res = float(np.linalg.norm(H @ X - X * w, axis=0).max())
    return {"seconds": dt, "iterations": it, "max_residual": res, "cores": os.cpu_count(),
            "kind": "oracle (numpy block Davidson, FP64)", "evals": w}


def replica_throughput(local_ms, steps, dim, world, device):
    """Whole-job throughput of `world` independent replicas (weak scaling: every
    rank builds the same workload).  After a barrier the slowest rank's time
    decides: value = world x steps x positions / max over ranks of the time.
    Returns (max_ms, value)."""
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    max_ms = float(t.item())
    return max_ms, world * steps * positions(dim) / (max_ms / 1000.0)


def run_reference(args, rank, world):
    from paper_1709_03005_gb300 import synth
    if rank != 0:
        return
    P = synth.make_config(args.config, **overrides(args))
    # each step is a bounded sample sized so that warm-up and steps together
    # take a few minutes
    budget = min(20.0, max(1.5, 60.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_baseline(P, budget)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(P, budget))
    dt = time.perf_counter() - t0
    v = float(np.mean([x["value"] for x in vals]))
    cb = dict(vals[-1])
    cb["value"] = v
    print(json.dumps({"metric": "H elements/sec", "value": v, "unit": "H elements/s", "n_gpus": args.gpus,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / max(args.steps, 1),
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "impl": "reference",
                      "config": {"workload": workload_text(args)},
                      "cpu_baseline": cb, "e2e": {"value": v, "unit": "H elements/s", "h2d_bytes_per_step": 0,
                                                  "d2h_bytes_per_step": 0}}), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1709_03005_gb300 import build_ext, hb, synth
    torch.cuda.set_device(local_rank)
    build_ext.build()
    precision = hb.HB_MIXED if args.precision == "mixed" else hb.HB_FP64
    P = synth.make_config(args.config, **overrides(args))
    dim = P.dim
    H = hb.Hamiltonian(P, validate=False)
    blocks = H.allocate()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def timed_builds(prec, steps, clock=None):
        times, st_list = [], []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, st = H.build(prec, blocks)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            st_list.append(st)
        return times, st_list

    for _ in range(args.warmup):
        H.build(precision, blocks)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        times, sts = timed_builds(precision, args.steps)
        torch.cuda.synchronize()
    total_ms, value = replica_throughput(float(np.sum(times)), args.steps, dim, world, "cuda")
    st = sts[-1]
    launches = sum(x.kernel_launches for x in sts)
    gemm_ms = float(np.mean([x.ms_expand_gemm for x in sts]))
    exp_ms = float(np.mean([x.ms_expand for x in sts]))

    # the sharded build (Section 3.1), with --sharded: every rank contracts its
    # share of the bra determinants, an all-reduce (NCCL under torchrun) sums
    # the partial coefficient rows, and every rank expands its share of the
    # tiles and L2 rows.  The total work is one build for any number of ranks
    # (strong scaling): the value is one build's positions over the slowest
    # rank's time per step.
    sharded = None
    if args.sharded:
        import torch.distributed as dist
        part = torch.empty(max(H.shard_coef_len(), 1), dtype=torch.float64, device="cuda")
        sb = H.allocate()

        def sharded_step():
            partial, _ = H.build_contract(precision, rank, world, part)
            if world > 1:
                dist.all_reduce(partial, op=dist.ReduceOp.SUM)
            H.build_expand(precision, rank, world, partial, sb)

        for _ in range(args.warmup):
            sharded_step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ts = []
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sharded_step()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = torch.tensor([float(np.mean(ts))], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(ms, op=dist.ReduceOp.MAX)
        ms = float(ms.item())
        sharded = {"ranks": world, "scaling": "strong", "ms_per_step": ms, "value": positions(dim) / (ms / 1e3),
                   "unit": "H elements/s",
                   "exchange_bytes_per_step": 8 * H.shard_coef_len() if world > 1 else 0}
        del sb, part
        torch.cuda.empty_cache()

    # the plain FP64 GPU build of the same instance, after the timed steps
    fp64 = None
    if precision == hb.HB_MIXED and args.fp64_steps > 0:
        H.build(hb.HB_FP64, blocks)
        torch.cuda.synchronize()
        t64, s64 = timed_builds(hb.HB_FP64, args.fp64_steps)
        ms64 = float(np.mean(t64))
        fp64 = {"ms_per_step": ms64, "value": positions(dim) / (ms64 / 1e3), "unit": "H elements/s",
                "steps": args.fp64_steps, "expand_kernel_ms": float(np.mean([x.ms_expand_gemm for x in s64])),
                "stages_ms": {"target": s64[-1].ms_target, "expand": s64[-1].ms_expand,
                              "class4": s64[-1].ms_class4, "l2": s64[-1].ms_l2}}

    # end to end through the public API with host buffers: staging (H2D of the
    # problem from pinned host memory, hb_init), build, and the D2H read of
    # every block into pinned host memory, each step
    e2e_steps = max(1, min(args.steps, 3))
    Pp = pinned_problem(P)
    h2d = sum(np.asarray(a).nbytes for a in (P.h, P.eri_tttt, P.eri_tttc, P.eri_ttcc, P.eri_tctc, P.l2_dets)) + \
        sum(g.dets.nbytes + g.ci.nbytes for g in P.groups)
    host = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in blocks.items()}
    d2h = sum(v.numel() * v.element_size() for v in host.values())
    init_ms = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        t1 = time.perf_counter()
        H2 = hb.Hamiltonian(Pp, validate=False)
        torch.cuda.synchronize()
        init_ms.append(1e3 * (time.perf_counter() - t1))
        b2, _ = H2.build(precision)
        for k, v in b2.items():
            host[k].copy_(v, non_blocking=True)
        torch.cuda.synchronize()
        H2.close()
        del b2
    torch.cuda.synchronize()
    e2e_value = world * e2e_steps * positions(dim) / (time.perf_counter() - t0)
    del host

    peaks = measured_peaks()
    if precision == hb.HB_MIXED:
        kern_ms = gemm_ms
        tflops = st.expand_tensor_flops
        pk = peaks.get("bf16_tflops")
        fp64eq = st.expand_flops / (kern_ms / 1e3) / 1e12 if kern_ms else None
        pipe = tflops / (kern_ms / 1e3) / 1e12 if kern_ms else None
        roof = {"bound": "tensor", "unit": "TFLOP/s", "peak": pk,
                "peak_source": "measured bf16 burst (of measured)",
                "kernel": "split_expand_kernel: Eq. 7 contraction on bf16 tensor cores, 6 slices per operand",
                "achieved": fp64eq, "flops_per_launch": st.expand_flops,
                "flops_definition": "algorithmic FP64-equivalent flops 2 K (elements) of Eq. 7 per launch",
                "kernel_ms": kern_ms,
                "pipe_achieved": pipe, "pipe_frac": pipe / pk if pipe and pk else None,
                "pipe_flops_per_launch": tflops,
                "pipe_definition": "bf16 tensor flops issued: the 21 slice-pair products of every FP64-equivalent "
                                   "product",
                "traffic": profiled_traffic("split_expand_kernel", "paper_1709_03005_gb300/csrc/k_split.cu",
                                            None if args.set else args.config)}
    else:
        kern_ms = exp_ms
        roof = {"bound": "alu", "unit": "TFLOP/s", "peak": fp64_alu_peak_tflops(),
                "peak_source": "derived FP64 peak: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz",
                "kernel": "expand_fp64_kernel: Eq. 7 contraction in FP64",
                "achieved": st.expand_flops / (kern_ms / 1e3) / 1e12 if kern_ms else None,
                "flops_per_launch": st.expand_flops, "kernel_ms": kern_ms,
                "traffic": profiled_traffic("expand_fp64_kernel", "paper_1709_03005_gb300/csrc/k_expand.cu",
                                            None if args.set else args.config)}
    roof["frac"] = roof["achieved"] / roof["peak"] if roof["achieved"] and roof["peak"] else None
    try:
        roof_c4 = class4_roofline(int(H.layout.n_l2), int(H.layout.contracted_dim),
                                  float(np.mean([x.ms_class4_kernel for x in sts])), peaks)
    except Exception as e:      # a report field: never lose the bench line for it
        roof_c4 = {"error": str(e)}
    H.close()
    del blocks
    torch.cuda.empty_cache()

    # Davidson on the medium workload (lowest 20 eigenpairs): block products
    # on the tensor cores (split bf16) and in FP64 on the GPU, the CPU
    # baseline beside them
    davidson = None
    if args.davidson_k > 0:
        Pd = synth.make_config(args.davidson_config)
        Hd = hb.Hamiltonian(Pd, validate=False)
        bd, _ = Hd.build(hb.HB_MIXED)
        torch.cuda.synchronize()

        def solve(flags):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ev, dst, ok = Hd.diag(bd, args.davidson_k, 1e-8, 400, precond=hb.HB_PRECOND_DIAG | flags,
                                  allow_not_converged=True)
            torch.cuda.synchronize()
            return {"seconds": time.perf_counter() - t0, "iterations": dst.iterations, "converged": ok,
                    "max_residual": dst.max_residual, "matvec_ms": dst.ms_matvec, "rr_ms": dst.ms_rr,
                    "gram_ms": dst.ms_gram, "combine_ms": dst.ms_combine,
                    "fp64_projections": fp64_projection_rate(dst)}, ev
        try:
            davidson = {"workload": CONFIG_TEXT.get(args.davidson_config, args.davidson_config),
                        "k": args.davidson_k, "tol": 1e-8}
            davidson["tensor_products"], ev_t = solve(hb.HB_DIAG_TENSOR)
            davidson["fp64_products"], ev_f = solve(0)
            if rank == 0 and args.cpu_baseline:
                cd = cpu_davidson(Pd, args.davidson_k)
                davidson["cpu_baseline"] = {k: v for k, v in cd.items() if k != "evals"}
                davidson["max_eval_diff_vs_cpu"] = float(np.abs(ev_t - cd["evals"]).max())
                davidson["speedup_vs_cpu"] = cd["seconds"] / davidson["tensor_products"]["seconds"]
        except hb.HBError as e:
            davidson = {"unavailable": str(e)}
        Hd.close()
        del bd
        torch.cuda.empty_cache()

    # the L2-heavy shape of the paper's H3PO4 run (contracted 712, 122103 L2
    # functions): the build and the lowest 20 eigenpairs
    l2_heavy = None
    if args.l2_heavy:
        try:
            Pl = synth.make_config("h3po4")
            Hl = hb.Hamiltonian(Pl, validate=False)
            bl, _ = Hl.build(hb.HB_MIXED)
            torch.cuda.synchronize()
            tl = []
            for _ in range(3):
                flush.zero_()
                _, stl = Hl.build(hb.HB_MIXED, bl)
                tl.append(stl.ms_total)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ev, dst, ok = Hl.diag(bl, 20, 1e-8, 400, precond=hb.HB_PRECOND_DIAG | hb.HB_DIAG_TENSOR,
                                  allow_not_converged=True)
            torch.cuda.synchronize()
            l2_heavy = {"workload": "l2_heavy_h3po4: 50 target + 89 continuum orbitals, N=14+1, 2000 target dets, "
                                    "8 states, 122103 L2, dim 122815", "l2_nnz": int(Hl.layout.l2_nnz),
                        "build_ms": float(np.median(tl)), "value": positions(Hl.dim) / (np.median(tl) / 1e3),
                        "unit": "H elements/s",
                        "davidson": {"k": 20, "tol": 1e-8, "seconds": time.perf_counter() - t0,
                                     "iterations": dst.iterations, "fp64_iterations": dst.fp64_iterations,
                                     "converged": ok, "max_residual": dst.max_residual, "matvec_ms": dst.ms_matvec}}
            Hl.close()
            del bl
            torch.cuda.empty_cache()
        except hb.HBError as e:
            l2_heavy = {"unavailable": str(e)}

    # the learned-preconditioner workload: lowest 200 eigenpairs, dimension 60000
    davidson_c5 = None
    if args.c5_k > 0:
        try:
            P5 = synth.make_config("c5")
            H5 = hb.Hamiltonian(P5, validate=False)
            b5, st5 = H5.build(hb.HB_MIXED)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ev, dst, ok = H5.diag(b5, args.c5_k, 1e-8, 400, precond=hb.HB_PRECOND_DIAG | hb.HB_DIAG_TENSOR,
                                  allow_not_converged=True)
            torch.cuda.synchronize()
            davidson_c5 = {"workload": "c5_learned: 40 target + 400 continuum orbitals, N=14+1, 20000 target dets, "
                                       "50 states, 40000 L2, dim 60000", "k": args.c5_k, "tol": 1e-8,
                           "precond": "diagonal", "seconds": time.perf_counter() - t0, "iterations": dst.iterations,
                           "fp64_iterations": dst.fp64_iterations, "converged": ok,
                           "max_residual": dst.max_residual, "matvec_ms": dst.ms_matvec, "rr_ms": dst.ms_rr,
                           "gram_ms": dst.ms_gram, "combine_ms": dst.ms_combine,
                           "fp64_projections": fp64_projection_rate(dst)}
            H5.close()
            del b5
            torch.cuda.empty_cache()
        except hb.HBError as e:
            davidson_c5 = {"unavailable": str(e)}

    # the batched workload: 16 symmetry / spin-coupling Hamiltonians, one graph
    # launch; the plain FP64 batch is timed beside it for the speedup
    batched = None
    if args.batched:
        try:
            lo, hi = (int(x) for x in args.batched_cont.split(","))
            fam = synth.make_batched_family(cont_per_irrep=(lo, hi))
            res = {}
            for name, prec in (("mixed", hb.HB_MIXED), ("fp64", hb.HB_FP64)):
                B = hb.Batch(fam, prec)
                for _ in range(3):
                    B.launch(stats=False)
                torch.cuda.synchronize()
                bt, gm = [], []
                for _ in range(max(3, min(args.steps, 5))):
                    flush.zero_()
                    stb = B.launch()
                    bt.append(stb.ms_total)
                    gm.append(stb.ms_expand_gemm)
                res[name] = dict(ms=float(np.mean(bt)), gemm_ms=float(np.mean(gm)), st=stb, nodes=B.nodes,
                                 positions=B.positions, dims=[h.dim for h in B.hams], report=B.report())
                B.close()
            m, f = res["mixed"], res["fp64"]
            st_m = m["st"]
            ach = st_m.expand_tensor_flops / (m["gemm_ms"] / 1e3) / 1e12 if m["gemm_ms"] else None
            pk = measured_peaks().get("bf16_tflops")
            batched = {"workload": "16 Hamiltonians (8 irreps x 2 spin couplings), dims "
                                   f"{min(m['dims'])}-{max(m['dims'])}, shared integrals",
                       "value": m["positions"] / (m["ms"] / 1e3), "unit": "H elements/s",
                       "ms_per_launch": m["ms"], "fp64_ms_per_launch": f["ms"],
                       "speedup_vs_fp64_batch": f["ms"] / m["ms"],
                       "graph_nodes": m["nodes"], "graph_launches_per_step": 1,
                       "kernel_launches_per_graph": st_m.kernel_launches,
                       "stages_ms": {"target": st_m.ms_target, "expand": st_m.ms_expand,
                                     "class4": st_m.ms_class4, "l2": st_m.ms_l2, "expand_gemm": m["gemm_ms"]},
                       "roofline_split_kernel": {"bound": "tensor", "unit": "TFLOP/s", "achieved": ach, "peak": pk,
                                                 "frac": ach / pk if ach and pk else None,
                                                 "flops_per_launch": st_m.expand_tensor_flops},
                       "autotuned": m["report"][:160] + ("..." if len(m["report"]) > 160 else "")}
        except hb.HBError as e:
            batched = {"unavailable": str(e)}

    if rank == 0:
        cb = cpu_baseline(P) if args.cpu_baseline else None
        out = {"metric": "H elements/sec", "value": value, "unit": "H elements/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "bf16x6-split/f32->f64" if precision == hb.HB_MIXED else "f64", "data": "synthetic",
               "config": {"workload": workload_text(args), "dim": dim,
                          "positions": positions(dim), "l2_flush": "256 MB write between timed steps",
                          "parallelism": f"replicas x{world}", "precision": args.precision},
               "sharded": sharded, "fp64": fp64, "speedup_vs_fp64": fp64["ms_per_step"] / (total_ms / args.steps) if fp64 else None,
               "init_ms": float(np.mean(init_ms)),
               "roofline": roof, "roofline_class4": roof_c4, "cpu_baseline": cb,
               "e2e": {"value": e2e_value, "unit": "H elements/s", "h2d_bytes_per_step": int(h2d),
                       "d2h_bytes_per_step": int(d2h)},
               "gpu_launches": launches, "clocks": clk.summary(), "davidson": davidson, "davidson_c5": davidson_c5,
               "l2_heavy": l2_heavy, "batched": batched,
               "stages_ms": {"target": st.ms_target, "expand": st.ms_expand, "class4": st.ms_class4,
                             "class4_kernel": st.ms_class4_kernel, "l2": st.ms_l2, "expand_kernel": gemm_ms}}
        print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c3")
    ap.add_argument("--set", action="append", default=[], metavar="KEY=INT",
                    help="override an integer size of the workload (e.g. n_l2=4000), for small profiling cases")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--davidson-k", type=int, default=20)
    ap.add_argument("--davidson-config", default="c2")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--c5-k", type=int, default=200, help="eigenpairs of the dimension-60000 workload (0: skip)")
    ap.add_argument("--no-l2-heavy", dest="l2_heavy", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-batched", dest="batched", action="store_false")
    ap.add_argument("--batched-cont", default="50,400", metavar="LO,HI",
                    help="continuum orbitals per irrep of the batched workload (smaller for profiling)")
    ap.add_argument("--sharded", action="store_true",
                    help="also time the sharded build (contraction share, all-reduce, expansion share per rank)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
