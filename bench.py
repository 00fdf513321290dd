#!/usr/bin/env python3
"""Butterfly apply throughput on GB300: points x RHS per second.

Default workload: the 2-D generalized Radon analogue, N = 1024 (2^20 sources and
targets), q = 5 (r = 25), one right-hand side, mixed precision (complex64
weights, FP32 interpolation, double-float phase).  A step is one full apply
(init, 5 column levels, switch, 5 row levels, final) on inputs resident in HBM.

Printed (one JSON line on rank 0): value (points*RHS/s), the FP64 GPU butterfly
on the same problem and the speedup over it, relative errors against the FP64
oracle (restricted butterfly on one level-m target box, and the direct sum on
sampled targets), the roofline of the dominant kernel pass (timed live with CUDA
events on the launching stream), the end-to-end rate through the host-buffer C
ABI call, the CPU oracle baseline, SM clocks sampled during the timed region.

--impl reference times the FP64 CPU oracle (the only reference this method has).
Under torchrun every rank runs an independent replica (the single-problem path
has no data-parallel split here); value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "butterfly apply points*RHS/s at stated rel-err, mixed/batched vs FP64 GPU; %roof"
UNIT = "points*RHS/s"
FP32_LANES_PER_SM = 128

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of each pass of the default
# workload, from one ncu capture of `python bench.py --steps 1 --warmup 1 --no-cpu-baseline --no-accuracy
# --fp64-steps 0 --no-autotune --no-tables --no-batched` (the dominant pass writes 0.85 GB more than its
# weights: register spills of its switch at three CTAs per SM reach DRAM).  They describe the kernels as
# built from sources with the recorded hash and the recorded pass schedule; otherwise the figure is
# dropped (traffic: null) until captured again.
TRAFFIC = {"genradon2d": {"src_sha256": "dc76e76eb7bedb887e3406a09fcc93cc26f2fb4562519df8098120ea50debe0d",
                          "schedule": ["col2", "col3", "row2", "row3"],
                          "bytes": [161666560, 1272867328, 369475328, 215727104]}}
TRAFFIC_SRC = ("bf_device.cuh", "bf_inst.cuh")   # the pass kernels and their launch configuration


def measured_hbm_gbs():
    """HBM copy bandwidth measured on this machine (MEASURED_PEAKS.json), else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_src_sha256():
    """Hash of the pass kernels' code with comments and blank lines removed (a change to the
    code voids the recorded traffic; a change to a comment does not)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in TRAFFIC_SRC:
        with open(os.path.join(ROOT, "paper_1305_4650_gb300", "csrc", name)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        lines = [ln.rstrip() for ln in text.splitlines() if ln.strip()]
        h.update("\n".join(lines).encode())
    return h.hexdigest()


def recorded_traffic(workload_name, schedule, pass_index):
    rec = TRAFFIC.get(workload_name)
    if (rec is None or rec["bytes"] is None or rec["src_sha256"] != kernel_src_sha256()
            or rec["schedule"] != schedule or pass_index >= len(rec["bytes"])):
        return None
    return rec["bytes"][pass_index]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="genradon2d",
                    choices=["genradon2d", "genradon3d", "dft64", "hypradon512", "hypradon48", "cg1024",
                             "genradon2d_points"])
    ap.add_argument("--nrhs", type=int, default=1, help="right-hand sides per apply (single-problem workloads)")
    ap.add_argument("--precision", default="", choices=["", "mixed", "mixed_sfu", "bf16x3", "tf32x3", "fp64"],
                    help="override the workload's precision (single-problem workloads)")
    ap.add_argument("--L", type=int, default=0, help="override log2 N of a single-problem workload (small cases)")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default tile schedules")
    ap.add_argument("--no-tables", action="store_true", help="skip the phase-table variant")
    ap.add_argument("--no-batched", action="store_true",
                    help="default workload: skip the 48-problem batch record (FP32, BF16x3, FP64 forms)")
    ap.add_argument("--batch-fp64-steps", type=int, default=1, help="timed FP64 steps of that batch record")
    ap.add_argument("--tc-levels", action="store_true",
                    help="bf16x3: run the column merge levels on the tensor cores too (bf_params.tc_levels)")
    ap.add_argument("--sharded", action="store_true",
                    help="under torchrun: one problem split over the ranks (bf_apply_shard + one NCCL all-reduce "
                         "of the targets per step, strong scaling) instead of independent replicas")
    return ap.parse_args()


def workload(name, L=0):
    from paper_1305_4650_gb300 import workloads as wl
    if L:   # a smaller (or larger) case of the same family, e.g. for profiling
        return {"genradon2d": lambda: wl.genradon2d(L), "genradon3d": lambda: wl.genradon3d(L),
                "dft64": lambda: wl.dft64().with_(L=L, name=f"dft_N{1 << L}_q5"),
                "hypradon512": lambda: wl.hypradon(L)}[name]()
    return {"genradon2d": wl.genradon2d, "genradon3d": wl.genradon3d, "dft64": wl.dft64,
            "hypradon512": lambda: wl.hypradon(9)}[name]()


# ------------------------------------------------------------------ clocks

class Clocks:
    """nvidia-smi sampler (200 ms) running during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------- algorithmic work

def phase_ops(phase: str, d: int, q: int) -> float:
    """FP32-pipe operations of one e^{2 pi i Phi} in the mixed path, counted from the
    double-float formulas with the per-dimension split of Phi: the part of source
    coordinate 0 (evaluated per phase), the parts of coordinates >= 1 (shared by the q
    phases of a node row), the sum of parts (an ordered fast two-sum where the parts are
    non-negative), the final sqrt / mod-1 step, and 18 for the quadrant-reduced sincos
    (setup 4, sin 4, cos 3, quadrant 7: degree-7 and degree-6 minimax polynomials in r^2 with
    2 pi folded in).  The frac of a double-float product costs 5 (two FMAs for the nearest
    integer and the remainder, two for the cross terms)."""
    sincos = 18
    if phase == "dot":
        part, add, fin = 5, 1, 0
    elif phase == "genradon":
        part, add, fin = 9, 8, 12
    elif phase == "hypradon":
        part, add, fin = 4, 8, 12
    else:
        part, add, fin = 11, 9, 4
    return part + (d - 1) * part / q + add + fin + sincos


def nonzero_lagrange(q: int, node_kind: int, xi: float) -> int:
    """Number of the q one-dimensional Lagrange values l_t(xi) = prod_{k != t} (xi - z_k) / (z_t - z_k)
    that are non-zero in FP64, as the plan computes them (nodes on [-1/2, 1/2]:
    cos(j pi / (q - 1)) / 2 Chebyshev-Lobatto, or cos((2j + 1) pi / 2q) / 2): the kernels skip
    the nodes whose value is exactly zero."""
    import math
    z = [0.5 * math.cos(j * math.pi / (q - 1)) if node_kind == 0 else 0.5 * math.cos((2 * j + 1) * math.pi / (2 * q))
         for j in range(q)]
    n = 0
    for t in range(q):
        v = 1.0
        for k in range(q):
            if k != t:
                v *= (xi - z[k]) / (z[t] - z[k])
        n += v != 0.0
    return n


def pass_work(spec, ps, nrhs=1):
    """Algorithmic counts of one kernel pass: phase evaluations, complex x real MACs
    (interpolation), complex multiplies (modulation) and complex MACs (switch)."""
    d, q, r, P = spec.d, spec.q, spec.r, spec.npts
    nz_src = nonzero_lagrange(q, spec.node_kind, spec.src_off - 0.5) ** d
    nz_tgt = nonzero_lagrange(q, spec.node_kind, spec.tgt_off - 0.5) ** d
    per_level_ph = (2 ** d + 1) * r
    per_level_mac = (2 ** (d + 1) - 2) * q ** (d + 1)
    w = dict(phases=0, macs=0, cmuls=0, cmacs=0)
    w["phases"] += ps["k"] * per_level_ph * P
    w["cmuls"] += ps["k"] * per_level_ph * P * nrhs
    w["macs"] += ps["k"] * per_level_mac * P * nrhs
    if ps["init"]:
        w["phases"] += (1 + nz_src) * P
        w["cmuls"] += (1 + nz_src) * P * nrhs
    if ps["switch"]:
        if spec.phase in ("dot", "separable"):          # factorised switch: d sweeps of q x q matrices
            w["phases"] += d * q * q * P
            w["cmacs"] += d * q ** (d + 1) * P * nrhs
        else:
            w["phases"] += r * r * P
            w["cmacs"] += r * r * P * nrhs
    if ps["final"]:
        w["phases"] += (1 + nz_tgt) * P
        w["cmuls"] += (1 + nz_tgt) * P * nrhs
    return w


def work_ops(spec, w):
    return w["phases"] * phase_ops(spec.phase, spec.d, spec.q) + 2 * w["macs"] + 4 * w["cmuls"] + 4 * w["cmacs"]


# ---------------------------------------------------------------- our arm

def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_1305_4650_gb300 import bf, workloads as wl
    if world > 1:
        import torch.distributed as dist
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    spec = workload(args.workload, args.L)
    nrhs = args.nrhs
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    prec = args.precision or spec.precision
    plan = bf.Plan.from_spec(spec, max_nrhs=nrhs, precision=prec, tc_levels=args.tc_levels)
    tuned = None if args.no_autotune else round(plan.autotune(nrhs, reps=3), 4)   # plan time, not timed
    passes = plan.passes(nrhs)
    g_np = wl.source_values(spec, nrhs, plan.cdtype, seed=spec.seed + rank)
    g = torch.from_numpy(g_np).to(dev)
    f = torch.empty_like(g)

    # ---- timed region: K applies through the C ABI (device buffers); with --sharded under
    # torchrun each step is this rank's part (bf_apply_shard) and one all-reduce of the targets
    sharded = args.sharded and world > 1
    if sharded:
        from paper_1305_4650_gb300 import sharding
        shard_g = sharding.shard_bits(world, spec.d)
        step = lambda: (plan.apply_shard(g, shard_g, rank, f=f), dist.all_reduce(f))
    else:
        step = lambda: plan.apply(g, f)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local_rank) as clk:
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps)
    clocks = clk.summary()
    value = spec.npts * nrhs * (1 if sharded else world) / (ms * 1e-3)
    if sharded:
        plan.apply(g, f)                                  # the rest of the line measures the whole apply
        torch.cuda.synchronize()
    out_f = f.cpu().numpy()

    # ---- per-pass device times (same passes, events between launches on the same stream)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(passes) + 1)]
    tpass = [0.0] * len(passes)
    for _ in range(args.steps):
        evs[0].record(stream)
        for i in range(len(passes)):
            plan.apply_pass(i, g.data_ptr(), f.data_ptr(), nrhs, sptr)
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
        for i in range(len(passes)):
            tpass[i] += evs[i].elapsed_time(evs[i + 1]) / args.steps
    dom = max(range(len(passes)), key=lambda i: tpass[i])
    sched = [{"switch_tc": "sw", "col_tc": "ctc"}.get(p["kind"], p["kind"]) + str(p["k"]) for p in passes]
    wdom = pass_work(spec, passes[dom], nrhs)
    ops = work_ops(spec, wdom)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * FP32_LANES_PER_SM * 2.07e9 / 1e12           # FP32-pipe Tops/s at the 2070 MHz max clock
    peak_basis = f"{sms} SMs x 128 FP32 lanes x 2.07 GHz (derived, one FP32-pipe op per lane per clock)"
    fma64 = bf.measure_fma_rate(True)
    if prec == "fp64":                                        # the FP64 pipe bounds the FP64 path
        peak = fma64 / 2
        peak_basis = "measured FP64 FMA rate (bf_measure_fma_rate), one FP64 op per FMA"
    achieved = ops / (tpass[dom] * 1e-3) / 1e12
    roofline = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 2), "unit": "Tops/s",
                "frac": round(achieved / peak, 4), "traffic": None if args.L else recorded_traffic(args.workload, sched, dom),
                "kernel": f"pass{dom}:{passes[dom]['kind']} l0={passes[dom]['l0']} k={passes[dom]['k']}"
                          + (" +init" if passes[dom]["init"] else "") + (" +switch" if passes[dom]["switch"] else "")
                          + (" +final" if passes[dom]["final"] else ""),
                "kernel_ms": round(tpass[dom], 4), "share": round(tpass[dom] / sum(tpass), 4),
                "peak_basis": peak_basis,
                "pass_ms": [round(t, 4) for t in tpass]}
    all_ops = sum(work_ops(spec, pass_work(spec, p, nrhs)) for p in passes)
    roofline["apply_frac"] = round(all_ops / (ms * 1e-3) / 1e12 / peak, 4)
    roofline["measured_fma_tflops"] = {"fp32": round(bf.measure_fma_rate(False), 1),
                                       "fp32_packed_pairs": round(bf.measure_fma_rate(packed=True), 1),
                                       "fp64": round(fma64, 3)}
    if prec != "fp64" and spec.d == 2:   # the phase ceiling: phases from registers only (bf_measure_phase_rate)
        roofline["phase_ceiling_gphs"] = {"scalar": round(plan.phase_rate(False), 1),
                                          "paired": round(plan.phase_rate(True), 1)}

    # ---- FP64 GPU butterfly on the same problem (the baseline of the speedup)
    fp64 = None
    if prec != "fp64" and args.fp64_steps > 0:
        p64 = bf.Plan.from_spec(spec, max_nrhs=nrhs, precision="fp64")
        if not args.no_autotune:
            p64.autotune(nrhs, reps=1)
        g64 = g.to(torch.complex128)
        f64 = torch.empty_like(g64)
        p64.apply(g64, f64)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(args.fp64_steps):
            p64.apply(g64, f64)
        a1.record(stream)
        torch.cuda.synchronize()
        ms64 = max_over_ranks(a0.elapsed_time(a1) / args.fp64_steps)
        fp64 = {"value": spec.npts * nrhs * world / (ms64 * 1e-3), "ms_per_step": round(ms64, 3),
                "speedup_mixed_over_fp64": round(ms64 / ms, 2)}
        out64 = f64.cpu().numpy()
        p64.close()

    # ---- the same apply with the special-function-unit sincos (BF_PREC_MIXED_SFU)
    sfu = None
    if prec == "mixed":
        psf = bf.Plan.from_spec(spec, max_nrhs=nrhs, precision="mixed_sfu")
        if not args.no_autotune:
            psf.autotune(nrhs, reps=3)
        fsf = torch.empty_like(g)
        for _ in range(args.warmup):
            psf.apply(g, fsf)
        torch.cuda.synchronize()
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        for _ in range(args.steps):
            psf.apply(g, fsf)
        b1.record(stream)
        torch.cuda.synchronize()
        ms_sfu = max_over_ranks(b0.elapsed_time(b1) / args.steps)
        sfu = {"value": spec.npts * nrhs * world / (ms_sfu * 1e-3), "ms_per_step": round(ms_sfu, 4),
               "precision": "mixed_sfu (complex64, double-float phase, SFU sin/cos)"}
        out_sfu = fsf.cpu().numpy()
        psf.close()

    # ---- the sharded form on this GPU: the time of one rank's part of the apply when the
    # sources are split over G = 2, 4 ranks (bf_apply_shard; ranks do equal work), against the
    # whole apply; the exchange is one all-reduce of the targets (bytes stated, not timed here)
    shard_rec = None
    if spec.d >= 2 and not args.L and world == 1 and prec != "fp64":
        shard_rec = {"all_reduce_bytes_per_step": spec.npts * nrhs * (16 if prec == "fp64" else 8)}
        fs_ = torch.empty_like(g)
        for G, sg in ((2, 1), (4, 2)):
            for _ in range(2):
                plan.apply_shard(g, sg, G - 1, f=fs_)
            torch.cuda.synchronize()
            d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            d0.record(stream)
            for _ in range(args.steps):
                plan.apply_shard(g, sg, G - 1, f=fs_)
            d1.record(stream)
            torch.cuda.synchronize()
            t = d0.elapsed_time(d1) / args.steps
            shard_rec[f"ranks{G}"] = {"per_rank_ms": round(t, 4), "fraction_of_apply": round(t / ms, 4)}
        shard_rec["note"] = ("per-rank part on one GPU (rank G-1; the ranks' parts are the same size); merges below the "
                             "last level run on the rank's pairs, the last pass on all pairs")
        del fs_

    # ---- phase-table variants (every phase evaluated once at plan creation; the apply reads
    # the reduced phases (one RHS) or the factors (several) and evaluates no Phi)
    tables = None
    if prec == "mixed" and (spec.d == 2 or nrhs == 1) and not args.no_tables:
        for tprec in ("mixed", "mixed_sfu"):
            ptb = bf.Plan.from_spec(spec, max_nrhs=nrhs, precision=tprec, phase_tables=True)
            tinfo = ptb.table_info()
            ftb = torch.empty_like(g)
            for _ in range(args.warmup):
                ptb.apply(g, ftb)
            torch.cuda.synchronize()
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            for _ in range(args.steps):
                ptb.apply(g, ftb)
            c1.record(stream)
            torch.cuda.synchronize()
            ms_tb = max_over_ranks(c0.elapsed_time(c1) / args.steps)
            # bytes an apply must move: the table once, the weights in and out of every pass boundary
            moved = tinfo["bytes"] + 2 * max(len(passes) - 1, 1) * spec.npts * spec.r * 8 * nrhs
            hbm_peak = measured_hbm_gbs()
            rec = {"value": spec.npts * nrhs * world / (ms_tb * 1e-3), "ms_per_step": round(ms_tb, 4),
                   "table_gb": round(tinfo["bytes"] / 1e9, 3), "build_ms": round(tinfo["build_ms"], 2),
                   "table_read_gbs": round(tinfo["bytes"] / (ms_tb * 1e-3) / 1e9, 1),
                   "hbm": {"achieved_gbs": round(moved / (ms_tb * 1e-3) / 1e9, 1), "peak_gbs": hbm_peak[0],
                           "frac": round(moved / (ms_tb * 1e-3) / 1e9 / hbm_peak[0], 3), "peak_basis": hbm_peak[1]},
                   "form": ("reduced phases (float), single-RHS kernels" if nrhs == 1
                            else "complex factors, multi-RHS kernels (bulk copies)")}
            if tprec == "mixed":
                out_tb = ftb.cpu().numpy()
                tables = rec
                tables["note"] = "plan-time phase tables (Section 1.4 precompute trade-off); plan creation not timed"
            else:
                tables["sfu_sincos"] = rec
            ptb.close()
            del ftb

    # ---- end to end through the C ABI with host buffers (H2D + apply + D2H per step)
    gh = torch.from_numpy(g_np).pin_memory()
    fh = torch.empty_like(gh).pin_memory()
    for _ in range(2):
        plan.apply_host_ptr(gh.data_ptr(), fh.data_ptr(), nrhs, sptr)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        plan.apply_host_ptr(gh.data_ptr(), fh.data_ptr(), nrhs, sptr)
    t1 = time.perf_counter()
    barrier()
    ms_e2e = max_over_ranks((t1 - t0) * 1e3 / args.steps)
    nbytes = g_np.nbytes
    e2e = {"value": spec.npts * nrhs * world / (ms_e2e * 1e-3), "unit": UNIT, "ms_per_step": round(ms_e2e, 3),
           "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}

    # ---- accuracy against the oracle (rank 0)
    acc = None
    if rank == 0 and not args.no_accuracy:
        import oracle
        P = oracle.Problem(**spec.oracle_kwargs())
        box = (1 << (spec.d * spec.switch_level)) // 3
        g0 = g_np[0].astype(np.complex128)
        tg = oracle.restricted_targets(P, spec.switch_level, box)
        t0 = time.perf_counter()
        ref = oracle.butterfly(P, g0, restrict=(spec.switch_level, box))[tg]
        t_or = time.perf_counter() - t0
        rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
        samp = tg[:: max(1, len(tg) // 32)]
        direct = oracle.direct_sum(P, g0, targets=samp)
        pos = np.searchsorted(tg, samp) if np.all(np.diff(tg) > 0) else [list(tg).index(s) for s in samp]
        acc = {"rel_l2_vs_oracle_butterfly": rel(out_f[0][tg], ref),
               "rel_l2_vs_direct_sum": rel(out_f[0][samp], direct),
               "oracle_butterfly_vs_direct_sum": rel(ref[pos], direct),
               "sample": f"{len(tg)} targets of level-{spec.switch_level} box {box}; direct sum on {len(samp)}",
               "oracle_s": round(t_or, 2)}
        if fp64 is not None:
            fp64["rel_l2_vs_oracle_butterfly"] = rel(out64[0][tg], ref)
            fp64["rel_l2_vs_direct_sum"] = rel(out64[0][samp], direct)
        if tables is not None:
            tables["rel_l2_vs_oracle_butterfly"] = rel(out_tb[0][tg], ref)
        if sfu is not None:
            sfu["rel_l2_vs_oracle_butterfly"] = rel(out_sfu[0][tg], ref)
            sfu["rel_l2_vs_direct_sum"] = rel(out_sfu[0][samp], direct)

    # ---- CPU oracle baseline (rank 0 at N = 1): restricted butterfly on one level-1 target box,
    # which does 1/2^d of the apply's work and yields 1/2^d of the outputs
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_sample(spec, g_np[0])

    plan.close()

    # ---- the 48-problem hyperbolic Radon batch (many right-hand sides, uneven N): FP32 and
    # BF16x3 multi-RHS forms against the FP64 GPU butterfly of the same batch (default schedules)
    batched = None
    if args.workload == "genradon2d" and not args.L and not args.no_batched:
        batched = batch_eval(args, rank, world, dev, min(args.steps, 5), args.warmup, False, args.batch_fp64_steps,
                             not args.no_accuracy)
    # ---- the other workloads of the method, compact (rank 0): d = 3, and the adjoint with CGLS
    configs = None
    if args.workload == "genradon2d" and not args.L and not args.no_batched and rank == 0:
        configs = {"genradon3d": config3_record(min(args.steps, 10), args.warmup, not args.no_accuracy),
                   "adjoint_cg": config5_record(min(args.steps, 10), args.warmup)}
    if rank != 0:
        return None
    csize = 8 if prec != "fp64" else 16
    weight_gb = 2 * max(len(passes) - 1, 1) * spec.npts * spec.r * csize * nrhs / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True,
            "scaling": "strong" if sharded else "weak", "vs_baseline": None, "dtype": "c128" if prec == "fp64" else "c64",
            "data": "synthetic",
            "config": {"workload": spec.name, "d": spec.d, "N": spec.N, "q": spec.q, "r": spec.r,
                       "phase": spec.phase, "precision": prec, "nrhs": nrhs, "switch_level": spec.switch_level,
                       "arithmetic": {"fp64": "complex128 weights, FP64 phase and sincos",
                                      "mixed": "complex64 weights, FP32 interpolation; Phi in double-float FP32 (>= 44 "
                                               "bits) reduced mod 1, polynomial FP32 sincos",
                                      "mixed_sfu": "as mixed, sin/cos from the special-function unit",
                                      "bf16x3": "as mixed; with several RHS the switch on the tensor cores, BF16x3 "
                                                "products with FP32 accumulation",
                                      "tf32x3": "as mixed; with several RHS the switch on the tensor cores, TF32x3 "
                                                "products with FP32 accumulation"}[prec],
                       "passes": len(passes), "fuse_levels": plan_fuse(passes),
                       "schedule": sched,
                       "autotuned_ms": tuned,
                       "l2": (f"no flush: each step streams {weight_gb:.1f} GB of weights through the 129 MB L2"
                              if weight_gb > 0.2 else "no flush: the whole working set is L2-resident (small case)"),
                       "parallelism": (f"one problem over {world} ranks (source-box sharding + all-reduce)"
                                       if sharded else f"replicas x{world}")},
            "roofline": roofline, "fp64_gpu": fp64, "sfu_sincos": sfu, "phase_tables": tables, "accuracy": acc,
            "batched": batched, "configs": configs, "sharded": shard_rec, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": args.steps * len(passes), "clocks": clocks}
    return line


def batch_eval(args, rank, world, dev, steps, warmup, autotune, fp64_steps, accuracy):
    """The 48 hyperbolic Radon problems (16 each of N = 128, 256, 512; 1..16 RHS each, drawn
    from the seed), q = 5, in five forms on the same inputs:
      mixed_per_pass   FP32 multi-RHS kernels, one launch per pass of every problem (bf_apply_batched)
      mixed_persistent the same kernels as one persistent launch per step (bf_batch_apply)
      bf16x3_per_pass  the switch on the tensor cores (BF_PREC_BF16X3), one launch per pass
      tf32x3_per_pass  the switch on the tensor cores with TF32 parts (BF_PREC_TF32X3)
      fp64             the plain FP64 GPU butterfly (complex128), one launch per pass
    The first four are captured once in a CUDA graph and replayed; timed with CUDA events on
    the launching stream (max over ranks).  Under torchrun the problems are dealt round-robin
    to the ranks (independent problems, no exchange).  Accuracy (rank 0): the first problem of
    each N against the FP64 oracle butterfly (all outputs at N = 128, one level-m target box
    otherwise) and, on 32 targets of that box, against the direct sum."""
    import numpy as np
    import torch
    from paper_1305_4650_gb300 import bf, workloads as wl
    if world > 1:
        import torch.distributed as dist
    probs, _ = wl.hypradon_batch()
    mine = [(i, s, k) for i, (s, k) in enumerate(probs) if i % world == rank]
    nr = [k for _, _, k in mine]
    gs = [torch.from_numpy(wl.source_values(s, k, np.complex64, seed=s.seed + i)).to(dev) for i, s, k in mine]
    pts_rhs = sum(s.npts * k for s, k in probs)
    stream = torch.cuda.current_stream()
    samples = {}                                          # N -> index into mine (first problem of each N)
    for j, (_, s, _) in enumerate(mine):
        samples.setdefault(s.N, j)

    def max_over_ranks(t):
        if world == 1:
            return t
        tt = torch.tensor([t], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        return float(tt.item())

    def timed(fn, graph=True, n=steps, w=warmup):
        if graph:
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                for _ in range(2):                        # kernel attributes set before capture
                    fn(side)
            torch.cuda.current_stream().wait_stream(side)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                fn(None)
            run = g.replay
        else:
            run = lambda: fn(None)
        for _ in range(w):
            run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with Clocks(dev.index) as clk:
            if world > 1:
                dist.barrier()
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(n):
                run()
            e1.record(stream)
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
        return max_over_ranks(e0.elapsed_time(e1) / n), clk.summary()

    def make(prec):
        ps = []
        for (_, s, k) in mine:
            p = bf.Plan.from_spec(s, max_nrhs=k, precision=prec)
            if autotune and prec != "fp64":
                p.autotune(k, reps=2)                     # plan time, not timed
            ps.append(p)
        return ps

    forms, outs, launches = {}, {}, {}
    # FP32 multi-RHS: per-pass graph and the persistent kernel
    plans = make("mixed")
    fs = [torch.empty_like(g) for g in gs]
    ms, clk = timed(lambda st: bf.apply_batched(plans, gs, fs, nr, stream=st))
    forms["mixed_per_pass"] = {"ms_per_step": round(ms, 3), "value": pts_rhs / (ms * 1e-3), "clocks": clk,
                               "launches_per_step": sum(p.launches(k) for p, k in zip(plans, nr))}
    outs["mixed"] = [fs[j].cpu().numpy() for j in samples.values()]
    batch = bf.Batch(plans, nr)
    binfo = batch.info()
    ms, clk = timed(lambda st: batch.apply(gs, fs, stream=st))
    waits = batch.wait_stats()
    forms["mixed_persistent"] = {"ms_per_step": round(ms, 3), "value": pts_rhs / (ms * 1e-3), "clocks": clk,
                                 "launches_per_step": 1, "work_units": binfo["units"], "jobs": binfo["jobs"],
                                 "ctas": binfo["grid"], "wait_timed_out": batch.status(),
                                 "dependency_waits": waits["waits"]}
    batch.close()
    big = max((j for j in range(len(mine)) if mine[j][1].N == 512), key=lambda j: nr[j], default=None)
    for p in plans:
        p.close()
    # BF16x3: the switch on the tensor cores
    plans = make("bf16x3")
    ms, clk = timed(lambda st: bf.apply_batched(plans, gs, fs, nr, stream=st))
    forms["bf16x3_per_pass"] = {"ms_per_step": round(ms, 3), "value": pts_rhs / (ms * 1e-3), "clocks": clk,
                                "launches_per_step": sum(p.launches(k) for p, k in zip(plans, nr)),
                                "tc_wait_timed_out": any(p.table_info()["timed_out"] for p in plans)}
    outs["bf16x3"] = [fs[j].cpu().numpy() for j in samples.values()]
    # per-pass times of the largest N = 512 problem, both precisions (events between launches)
    roof = None
    if big is not None:
        roof = {}
        for prec in ("mixed", "bf16x3"):
            p = plans[big] if prec == "bf16x3" else bf.Plan.from_spec(mine[big][1], max_nrhs=nr[big], precision="mixed")
            if prec == "mixed" and autotune:
                p.autotune(nr[big], reps=2)
            roof[prec] = pass_roofline(p, mine[big][1], nr[big], gs[big], fs[big], stream, dev, steps)
            if prec == "mixed":
                p.close()
        roof["problem"] = f"N=512, {nr[big]} RHS"
    for p in plans:
        p.close()
    # TF32x3: the switch on the tensor cores with TF32 parts (the accuracy of the FP32 form)
    plans = make("tf32x3")
    ms, clk = timed(lambda st: bf.apply_batched(plans, gs, fs, nr, stream=st))
    forms["tf32x3_per_pass"] = {"ms_per_step": round(ms, 3), "value": pts_rhs / (ms * 1e-3), "clocks": clk,
                                "launches_per_step": sum(p.launches(k) for p, k in zip(plans, nr)),
                                "tc_wait_timed_out": any(p.table_info()["timed_out"] for p in plans)}
    outs["tf32x3"] = [fs[j].cpu().numpy() for j in samples.values()]
    for p in plans:
        p.close()
    del fs
    # FP64 GPU butterfly of the same batch
    if fp64_steps > 0:
        plans = make("fp64")
        g64 = [g.to(torch.complex128) for g in gs]
        f64 = [torch.empty_like(g) for g in g64]
        ms, clk = timed(lambda st: bf.apply_batched(plans, g64, f64, nr, stream=st), graph=False, n=fp64_steps, w=1)
        forms["fp64_per_pass"] = {"ms_per_step": round(ms, 3), "value": pts_rhs / (ms * 1e-3), "clocks": clk,
                                  "steps": fp64_steps}
        outs["fp64"] = [f64[j].cpu().numpy() for j in samples.values()]
        for p in plans:
            p.close()
        del g64, f64
    acc = None
    if rank == 0 and accuracy:
        import oracle
        rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
        acc = {}
        for n_i, (N, j) in enumerate(samples.items()):
            i0, s0, k0 = mine[j]
            P = oracle.Problem(**s0.oracle_kwargs())
            g0 = gs[j].cpu().numpy().astype(np.complex128)
            lvl = s0.switch_level
            box = (1 << (2 * lvl)) // 3
            tg = np.arange(s0.npts) if N == 128 else oracle.restricted_targets(P, lvl, box)
            rhs = list(range(k0)) if N == 128 else [0]
            ref = [oracle.butterfly(P, g0[r]) if N == 128 else oracle.butterfly(P, g0[r], restrict=(lvl, box))
                   for r in rhs]
            samp = tg[:: max(1, len(tg) // 32)][:32]
            direct = oracle.direct_sum(P, g0[0], targets=samp)
            rec = {"problem": i0, "nrhs": k0,
                   "compared": "all outputs, every RHS" if N == 128 else f"level-{lvl} target box {box}, RHS 0",
                   "oracle_vs_direct_sum": rel(ref[0][samp], direct)}
            for arm, o in outs.items():
                out = o[n_i]
                rec[arm] = {"rel_l2_vs_oracle_butterfly": max(rel(out[r][tg], ref[x][tg]) for x, r in enumerate(rhs)),
                            "rel_l2_vs_direct_sum": rel(out[0][samp], direct)}
            acc[f"N{N}"] = rec
    fast = min(("mixed_per_pass", "mixed_persistent", "bf16x3_per_pass", "tf32x3_per_pass"),
               key=lambda f: forms[f]["ms_per_step"])
    rec = {"workload": "hypradon48_q5", "problems": len(probs), "N": [128, 256, 512],
           "nrhs_total": int(sum(k for _, k in probs)), "points_rhs": pts_rhs,
           "value": forms[fast]["value"], "unit": UNIT, "ms_per_step": forms[fast]["ms_per_step"], "form": fast,
           "forms": forms, "roofline": roof, "accuracy": acc,
           "schedules": "autotuned" if autotune else "default"}
    if "fp64_per_pass" in forms:
        rec["speedup_over_fp64"] = round(forms["fp64_per_pass"]["ms_per_step"] / forms[fast]["ms_per_step"], 2)
        rec["speedup_mixed_over_fp64"] = round(forms["fp64_per_pass"]["ms_per_step"] /
                                               forms["mixed_per_pass"]["ms_per_step"], 2)
    return rec


def timed_apply(fn, stream, steps, warmup):
    """ms per call of fn() on the launching stream (CUDA events, synchronised both sides)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def config3_record(steps, warmup, accuracy):
    """The d = 3 generalized Radon workload (N = 64, q = 4, 2^18 points): mixed and FP64 GPU
    applies, the speedup, and both against the oracle (one level-m box) and the direct sum."""
    import numpy as np
    import torch
    from paper_1305_4650_gb300 import bf, workloads as wl
    spec = wl.genradon3d()
    stream = torch.cuda.current_stream()
    rec, outs = {"workload": spec.name, "points": spec.npts}, {}
    g32 = wl.source_values(spec, 1, np.complex64)
    for prec, n in (("mixed", steps), ("fp64", max(1, steps // 5))):
        g_np = g32.astype(np.complex128) if prec == "fp64" else g32
        plan = bf.Plan.from_spec(spec, precision=prec)
        plan.autotune(1, reps=2)
        g = torch.from_numpy(g_np).cuda()
        f = torch.empty_like(g)
        ms = timed_apply(lambda: plan.apply(g, f), stream, n, 2)
        rec[prec] = {"ms_per_step": round(ms, 3), "value": spec.npts / (ms * 1e-3), "launches": plan.launches(1)}
        outs[prec] = (g_np[0], f.cpu().numpy()[0])
        plan.close()
    rec["speedup_mixed_over_fp64"] = round(rec["fp64"]["ms_per_step"] / rec["mixed"]["ms_per_step"], 2)
    # the plan-time phase table (the reduced phase of every factor, one float each) against the
    # evaluating apply of the same schedule: time, bytes moved, and bit-identical results
    hbm_peak = measured_hbm_gbs()
    rec["phase_tables"] = {}
    for tprec in ("mixed", "mixed_sfu"):
        pt = bf.Plan.from_spec(spec, precision=tprec, phase_tables=True)
        pe = bf.Plan.from_spec(spec, precision=tprec)
        g = torch.from_numpy(g32).cuda()
        ft, fe = torch.empty_like(g), torch.empty_like(g)
        ms_t = timed_apply(lambda: pt.apply(g, ft), stream, steps, 2)
        ms_e = timed_apply(lambda: pe.apply(g, fe), stream, steps, 2)
        torch.cuda.synchronize()
        info = pt.table_info()
        moved = info["bytes"] + 2 * max(len(pt.passes(1)) - 1, 1) * spec.npts * spec.r * 8
        rec["phase_tables"][tprec] = {
            "ms_per_step": round(ms_t, 3), "value": spec.npts / (ms_t * 1e-3),
            "evaluating_ms_per_step": round(ms_e, 3), "speedup_over_evaluating": round(ms_e / ms_t, 2),
            "table_gb": round(info["bytes"] / 1e9, 3), "build_ms": round(info["build_ms"], 2),
            "bit_identical_to_evaluating": bool(torch.equal(ft, fe)), "timed_out": bool(info["timed_out"]),
            "hbm": {"achieved_gbs": round(moved / (ms_t * 1e-3) / 1e9, 1), "peak_gbs": hbm_peak[0],
                    "frac": round(moved / (ms_t * 1e-3) / 1e9 / hbm_peak[0], 3), "peak_basis": hbm_peak[1]}}
        pt.close()
        pe.close()
        del g, ft, fe
    if accuracy:
        import oracle
        rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
        P = oracle.Problem(**spec.oracle_kwargs())
        lvl, box = spec.switch_level, 300
        tg = oracle.restricted_targets(P, lvl, box)
        g0 = outs["mixed"][0].astype(np.complex128)
        ref = oracle.butterfly(P, g0, restrict=(lvl, box))[tg]
        samp = tg[:: max(1, len(tg) // 32)][:32]
        direct = oracle.direct_sum(P, g0, targets=samp)
        where = {int(t): i for i, t in enumerate(tg)}      # tg is in Morton order, not sorted
        pos = np.array([where[int(t)] for t in samp])
        for prec in ("mixed", "fp64"):
            out = outs[prec][1]
            rec[prec]["rel_l2_vs_oracle_butterfly"] = rel(out[tg], ref)
            rec[prec]["rel_l2_vs_direct_sum"] = rel(out[samp], direct)
        rec["oracle_vs_direct_sum"] = rel(ref[pos], direct)
        rec["sample"] = f"{len(tg)} targets of level-{lvl} box {box}; direct sum on 32 (the FP64 arm's input is the mixed arm's, widened)"
    return rec


def config5_record(steps, warmup):
    """The adjoint workload (d = 2 generalized Radon, N = 1024, q = 5, mixed): the adjoint apply,
    the dot-product identity <B g, h> = <g, B^H h> at full size, and 20 CGLS iterations on
    B^H B m = B^H d with d = B m_true (1% spikes)."""
    import numpy as np
    import torch
    from paper_1305_4650_gb300 import bf, workloads as wl
    from paper_1305_4650_gb300.autograd import cgls
    spec = wl.genradon2d()
    stream = torch.cuda.current_stream()
    plan = bf.Plan.from_spec(spec, precision="mixed")
    plan.autotune(1, reps=2)
    g = torch.from_numpy(wl.source_values(spec, 1, np.complex64, seed=11)).cuda()
    h = torch.from_numpy(wl.source_values(spec, 1, np.complex64, seed=12)).cuda()
    gh = torch.empty_like(g)
    ms_adj = timed_apply(lambda: plan.apply_adjoint(h, gh), stream, steps, warmup)
    Bg = plan.apply(g)
    BHh = plan.apply_adjoint(h)
    c128 = lambda t: t.flatten().to(torch.complex128)
    lhs, rhs = torch.vdot(c128(h), c128(Bg)), torch.vdot(c128(BHh), c128(g))
    dot_err = (abs(lhs - rhs) / (torch.linalg.vector_norm(c128(Bg)) * torch.linalg.vector_norm(c128(h)))).item()
    mt = torch.from_numpy(wl.sparse_spikes(spec, 0.01)).cuda()
    d = plan.apply(mt)
    cgls(plan, d, 2)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    m, hist = cgls(plan, d, 20)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_cg = e0.elapsed_time(e1)
    plan.close()
    return {"workload": "cg20_" + spec.name, "adjoint_ms_per_apply": round(ms_adj, 3),
            "adjoint_value": spec.npts / (ms_adj * 1e-3), "dot_product_identity_rel": dot_err,
            "cg_iterations": 20, "cg_ms": round(ms_cg, 2), "cg_applies": 41,
            "cg_points_per_s": 41 * spec.npts / (ms_cg * 1e-3),
            "residual_history": [round(x / hist[0], 6) for x in hist[::4]] + [round(hist[-1] / hist[0], 6)],
            "residual_monotone": all(b <= a * (1 + 1e-6) for a, b in zip(hist, hist[1:]))}


def pass_roofline(plan, spec, nrhs, g, f, stream, dev, steps):
    """Per-pass device times of one apply (events between the launches on the launching
    stream) and the dominant pass against the FP32-lane peak: algorithmic FP32-pipe work
    (phases, interpolation, modulation; the switch's MACs too unless they run on the tensor
    cores) over its time."""
    import torch
    passes = plan.passes(nrhs)
    sptr = stream.cuda_stream
    for i in range(len(passes)):
        plan.apply_pass(i, g.data_ptr(), f.data_ptr(), nrhs, sptr)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(passes) + 1)]
    tp = [0.0] * len(passes)
    for _ in range(steps):
        evs[0].record(stream)
        for i in range(len(passes)):
            plan.apply_pass(i, g.data_ptr(), f.data_ptr(), nrhs, sptr)
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
        for i in range(len(passes)):
            tp[i] += evs[i].elapsed_time(evs[i + 1]) / steps
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * FP32_LANES_PER_SM * 2.07e9 / 1e12

    def alu_ops(ps):
        w = pass_work(spec, ps, nrhs)
        if ps["kind"] == "switch_tc":                 # the switch's MACs run on the tensor cores
            w = dict(w, cmacs=0)
        if ps["kind"] == "col_tc":                    # and so does this level's interpolation
            w = dict(w, macs=0)
        return work_ops(spec, w)

    dom = max(range(len(passes)), key=lambda i: tp[i])
    ops = alu_ops(passes[dom])
    return {"bound": "alu", "pass_ms": [round(t, 4) for t in tp],
            "schedule": [{"switch_tc": "sw", "col_tc": "ctc"}.get(p["kind"], p["kind"]) + str(p["k"]) for p in passes],
            "dominant": dom, "achieved": round(ops / (tp[dom] * 1e-3) / 1e12, 3), "peak": round(peak, 2),
            "unit": "Tops/s", "frac": round(ops / (tp[dom] * 1e-3) / 1e12 / peak, 4),
            "apply_frac": round(sum(alu_ops(p) for p in passes) / (sum(tp) * 1e-3) / 1e12 / peak, 4)}


def run_batched(args, rank, world, local_rank):
    """The 48-problem hyperbolic Radon batch as the line's workload (see batch_eval)."""
    import torch
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    rec = batch_eval(args, rank, world, dev, args.steps, args.warmup, not args.no_autotune, args.fp64_steps,
                     not args.no_accuracy)
    if rank != 0:
        return None
    fast = rec["forms"][rec["form"]]
    return {"metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": rec["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": "hypradon48_q5", "problems": rec["problems"], "N": rec["N"],
                       "nrhs_total": rec["nrhs_total"], "points_rhs": rec["points_rhs"], "form": rec["form"],
                       "precision": "bf16x3 (tensor-core switch) or mixed, the faster",
                       "l2": "no flush: each step streams ~20 GB of weights through the 129 MB L2",
                       "parallelism": f"problems round-robin over {world} rank(s)"},
            "batched": rec, "gpu_launches": args.steps * fast["launches_per_step"], "clocks": fast["clocks"]}


def run_cg(args, rank, world, local_rank):
    """20 CGLS iterations on B^H B m = B^H d, d = B m_true (1% spikes), generalized Radon
    N = 1024, q = 5, mixed: each iteration is one forward and one adjoint apply plus vector
    updates.  value = applies * N^d / time; the residual history is reported."""
    import numpy as np
    import torch
    from paper_1305_4650_gb300 import bf, workloads as wl
    from paper_1305_4650_gb300.autograd import cgls
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    spec = wl.genradon2d()
    plan = bf.Plan.from_spec(spec, precision="mixed")
    if not args.no_autotune:
        plan.autotune(1, reps=3)
    launches = plan.launches(1)
    mt = torch.from_numpy(wl.sparse_spikes(spec, 0.01)).to(dev)
    d = plan.apply(mt)
    iters = 20
    for _ in range(max(1, args.warmup // 3)):
        cgls(plan, d, 2)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local_rank) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        m, hist = cgls(plan, d, iters)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    applies = 2 * iters + 1
    plan.close()
    if rank != 0:
        return None
    return {"metric": METRIC, "value": applies * spec.npts * world / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": 1, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": "cg20_genradon2d_N1024_q5", "iterations": iters, "applies": applies,
                       "m_true": "1% spikes, N(0,1) amplitudes", "precision": "mixed"},
            "residual_history": [round(h / hist[0], 6) for h in hist],
            "gpu_launches": applies * launches,
            "clocks": clk.summary()}


def run_points(args, rank, world, local_rank):
    """2^20 sources and 2^20 targets at random positions (70% of each clustered in a small
    square, so many leaf boxes are empty and some crowded) for the generalized Radon phase
    with the N = 1024 box trees, q = 5, mixed.  value = 2^20 targets x RHS / time; error of
    32 sampled targets against the direct sum over all sources."""
    import numpy as np
    import torch
    from paper_1305_4650_gb300 import bf, workloads as wl
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    spec = wl.genradon2d(args.L or 10)
    n = spec.npts
    rng = np.random.default_rng(spec.seed + 7)
    x_lo, x_w, y_lo, y_w = spec.domain()

    def pts(lo, w):
        u = rng.random((n, 2))
        u = np.where(rng.random((n, 1)) < 0.7, 0.4 + 0.05 * u, u)
        return np.asarray(lo[:2]) + u * np.asarray(w[:2])

    y, x = pts(y_lo, y_w), pts(x_lo, x_w)
    t0 = time.perf_counter()
    plan = bf.Plan.from_spec(spec, precision="mixed", sources=y, targets=x)
    plan_s = time.perf_counter() - t0
    g_np = wl.source_values(spec, 1, np.complex64, seed=spec.seed + rank)
    g = torch.from_numpy(g_np).to(dev)
    f = plan.apply(g)
    for _ in range(args.warmup):
        plan.apply(g, f)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local_rank) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            plan.apply(g, f)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    acc = None
    if rank == 0 and not args.no_accuracy:
        import oracle
        P = oracle.Problem(**spec.oracle_kwargs())
        samp = rng.choice(n, 32, replace=False)
        ref = oracle.direct_sum_points(P, y, g_np[0].astype(np.complex128), x[samp])
        out = f.cpu().numpy()[0][samp]
        acc = {"rel_l2_vs_direct_sum": float(np.linalg.norm(out - ref) / np.linalg.norm(ref)),
               "sample": "32 random targets, direct sum over all 2^20 sources"}
    launches = plan.launches(1)
    plan.close()
    if rank != 0:
        return None
    return {"metric": METRIC, "value": n * world / (ms * 1e-3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": f"genradon2d_points_{n}", "d": 2, "tree_N": spec.N, "q": 5, "sources": n,
                       "targets": n, "placement": "70% clustered in 5% of each domain's width, rest uniform",
                       "precision": "mixed", "plan_s": round(plan_s, 2),
                       "parallelism": f"replicas x{world}"},
            "accuracy": acc, "gpu_launches": args.steps * launches, "clocks": clk.summary()}


def plan_fuse(passes):
    return max(p["k"] for p in passes)


def restricted_work_fraction(d: int, L: int, level: int) -> float:
    """Share of the apply's translations done by the oracle restricted to one target box at
    `level`: stage l touches the pairs whose target box lies on the box's path, and of their
    2^d children only those on the path (exactly 1/2^(d level) when level <= 1)."""
    tot = 0.0
    for l in range(L):
        act_pairs = 2.0 ** (-d * min(l, level))             # active target boxes at level l
        act_child = 2.0 ** (-d) if l < level else 1.0        # active children of each
        tot += act_pairs * act_child
    return tot / L


def cpu_sample(spec, g0, level=1):
    import numpy as np
    import oracle
    P = oracle.Problem(**spec.oracle_kwargs())
    box = 0
    n_out = spec.npts >> (spec.d * level)
    t0 = time.perf_counter()
    oracle.butterfly(P, np.asarray(g0, np.complex128), restrict=(level, box))
    dt = time.perf_counter() - t0
    frac = restricted_work_fraction(spec.d, spec.L, level)
    return {"value": n_out / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "seconds": round(dt, 2),
            "sample": f"FP64 oracle butterfly restricted to target box {box} at level {level}: "
                      f"{n_out} of {spec.npts} outputs, {frac:.4f} of the apply's translations "
                      f"(value = outputs / time)"}


# ---------------------------------------------------------- reference arm

def run_reference(args, rank, world):
    if rank != 0:
        return None
    import numpy as np
    import oracle
    from paper_1305_4650_gb300 import workloads as wl
    spec = workload(args.workload)
    g0 = wl.source_values(spec, 1, np.complex64)[0]
    level = 1
    for _ in range(args.warmup):
        cpu_sample(spec, g0, level)
    vals, secs = [], []
    for _ in range(args.steps):
        s = cpu_sample(spec, g0, level)
        vals.append(s["value"])
        secs.append(s["seconds"])
    value = len(vals) / sum(1.0 / v for v in vals)
    n_out = spec.npts >> (spec.d * level)
    ms = n_out / value * 1e3
    cpu = {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
           "sample": s["sample"]}
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": spec.name, "d": spec.d, "N": spec.N, "q": spec.q, "phase": spec.phase,
                       "precision": "fp64 (CPU oracle)", "nrhs": 1},
            "cpu_baseline": cpu, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                         "d2h_bytes_per_step": 0},
            "gpu_launches": 0}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
        runner = {"hypradon48": run_batched, "cg1024": run_cg, "genradon2d_points": run_points}.get(args.workload,
                                                                                                   run_ours)
        line = runner(args, rank, world, local_rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
