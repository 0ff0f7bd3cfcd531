#!/usr/bin/env python
"""Parallel-iDMRG benchmark on GB300: unit-cell steps per second.

A step is one parallel iteration n (Sec. 3): the l/2 two-site superblocks
of the unit cell are solved (Lanczos on H_eff psi), truncated by SVD and
renormalised, all through the C ABI of libidmrg.  Workload: S=1/2 random-bond
Heisenberg chain, l = 16 (8 superblocks per step), J_k ~ U[0.5, 1.5] from
PCG64 seed 1606, m = 256, measured in the saturated regime (D = m).

The headline is the mixed-precision path (H_eff psi on the tensor cores in
TF32x3, Lanczos and SVD in FP64); the same run times the FP64 path on the
same workload and reports the largest |dE/site| between the two.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec tf32x3|bf16x3|fp64|fp64tc] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun each rank runs its own
disorder realisation (seed 1606 + rank): independent problems, no exchange.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "iDMRG unit-cell steps/sec and H_eff·ψ TFLOP/s (mixed vs FP64) at |ΔE/site|≤1e-8"
WORKLOAD = "randchain_l16_m256"
SATURATE = 11            # iterations until every block holds m states (n >= log2 m + 2)
FLUSH_BYTES = 256 << 20  # > 129 MB L2
HBM_FALLBACK, BF16_FALLBACK, BF16_SUST_FALLBACK = 6800.0, 1900.0, 1700.0
FP64_ALU_PEAK = 152 * 2070e6 * 4 / 1e9   # GFLOP/s: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz


def peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return {"hbm": p["hbm_gbs"], "bf16": p["bf16_tflops"],
                "bf16_sustained": p.get("bf16_tflops_sustained", p["bf16_tflops"]), "src": "measured"}
    except Exception:
        return {"hbm": HBM_FALLBACK, "bf16": BF16_FALLBACK, "bf16_sustained": BF16_SUST_FALLBACK, "src": "fallback"}


def rank_seed(rank: int) -> int:
    """Disorder realisation of a rank: independent problems, one per GPU."""
    return 1606 + rank


def make_workload(rank: int, name: str = WORKLOAD):
    """The MPO of a named workload; the random-bond chain draws its couplings
    from the rank's seed (independent realisations), the cylinder is fixed."""
    from workloads import build_mpo, make_config, random_chain_bonds
    if name == WORKLOAD:
        seed = rank_seed(rank)
        return build_mpo(random_chain_bonds(16, 0.5, 1.5, seed), 16), seed
    mpo, _ = make_config(name)
    return mpo, None


def job_value(world: int, steps: int, seconds: float) -> float:
    """Whole-job throughput: every rank ran `steps` steps of its own problem;
    `seconds` is the slowest rank's time."""
    return world * steps / seconds


def reduce_max(values, dist, device):
    """Max over ranks of a few timings (the job takes as long as its slowest rank)."""
    import torch
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.p = None
        self.index = index

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out = self.p.communicate(timeout=5)[0]
        except Exception:
            self.p.kill()
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except ValueError:
                continue
            for name, v in zip(names, f[4:8]):
                if v.lower() in ("active", "1", "0x1"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def source_hash(*names):
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_1606_06790_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


KERNEL_SOURCES = {"heff_gemm": ["kernels_f64.cu", "kernels_tc.cu"], "heff_wstage": ["kernels_f64.cu", "kernels_tc.cu"],
                  "lanczos_vec": ["kernels_lanczos.cu"], "lanczos_tri": ["kernels_lanczos.cu"],
                  "svd": ["kernels_svd.cu", "kernels_tc.cu"], "env": ["kernels_f64.cu", "kernels_tc.cu"],
                  "predict": ["kernels_f64.cu", "kernels_tc.cu"], "heff_f64": ["kernels_f64.cu", "kernels_tc.cu"]}


def traffic_for(kclass: str, prec: str):
    """DRAM bytes per launch of a kernel class from a committed ncu summary
    (profiles/traffic.json), used only while the class's sources are unchanged."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        e = t[f"{kclass}/{prec}"]
        if e.get("source_hash") == source_hash(*KERNEL_SOURCES[kclass]):
            return e["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


def class_roofline(name: str, d: dict, prec: str, pk: dict):
    """Roofline of one kernel class from its event-timed launches.

    FP64 arithmetic (SVD, FP64 H_eff, environments, prediction) is bound by
    the FP64 units: 152 SMs x 2 FMA/clk x 2.07 GHz; the reduced-precision
    H_eff by the tensor pipe of its split type (measured sustained bf16, times
    the nominal tf32/bf16 ratio for TF32); the Lanczos vector kernels by HBM
    bandwidth."""
    sec = d["ms"] * 1e-3
    out = {"kernel": name, "launch_ms": d["ms"] / max(d["launches"], 1), "traffic": traffic_for(name, prec)}
    if name in ("heff_gemm", "heff_wstage") and prec != "fp64":
        bf = prec in ("bf16x3", "fp64tc")
        peak = pk["bf16_sustained"] * (1.0 if bf else 1.1 / 2.25)
        achieved = d["flops"] / sec / 1e12 if sec > 0 else 0.0
        src = "sustained bf16" if bf else "sustained bf16 x nominal tf32/bf16 (1.1/2.25)"
        what = ("FP64 products counted once (36 BF16 digit products each)" if prec == "fp64tc"
                else "split products counted once")
        out.update({"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "peak_source": f"{pk['src']} {src}; {what}"})
    elif name in ("heff_gemm", "heff_wstage", "heff_f64", "svd", "env", "predict"):
        achieved = d["flops"] / sec / 1e9 if sec > 0 else 0.0
        out.update({"bound": "alu", "achieved": achieved, "peak": FP64_ALU_PEAK, "unit": "GFLOP/s",
                    "peak_source": "FP64 FMA issue: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz"})
    else:
        achieved = d["bytes"] / sec / 1e9 if sec > 0 else 0.0
        out.update({"bound": "hbm", "achieved": achieved, "peak": pk["hbm"], "unit": "GB/s",
                    "peak_source": f"{pk['src']} copy bandwidth"})
    out["frac"] = out["achieved"] / out["peak"]
    keys = ("bound", "achieved", "peak", "unit", "frac", "traffic", "kernel", "launch_ms", "peak_source")
    return {k: out[k] for k in keys}


def heff_roofline(prof: dict, prec: str, pk: dict):
    """H_eff psi as a whole (GEMM stages + two-site MPO stage): the metric's FLOP/s."""
    d = {"ms": prof["heff_gemm"]["ms"] + prof["heff_wstage"]["ms"], "launches": prof["heff_gemm"]["launches"],
         "flops": prof["heff_gemm"]["flops"] + prof["heff_wstage"]["flops"], "bytes": 0.0}
    r = class_roofline("heff_gemm", d, prec, pk)
    r["kernel"] = "heff (gemm + wstage)"
    r["traffic"] = None
    return r


def cpu_baseline(mpo, m: int, budget_s: float = 25.0, timed_steps: int = 2):
    """The FP64 oracle as it stands on this host's cores: iterate from n = 1
    (untimed) into the saturated regime, then time up to `timed_steps` steps."""
    from oracle.idmrg import ParallelIDMRG
    cores = len(os.sched_getaffinity(0))
    ref = ParallelIDMRG.from_mpo(mpo, m=m)
    t0 = time.perf_counter()
    while ref.n <= SATURATE:
        ref.step()
        if time.perf_counter() - t0 > 4 * budget_s:
            break
    times = []
    for _ in range(timed_steps):
        t = time.perf_counter()
        ref.step()
        times.append(time.perf_counter() - t)
        if sum(times) > budget_s:
            break
    per = sum(times) / len(times)
    return ref, {"value": 1.0 / per, "unit": "unit-cell steps/s", "cores": cores, "kind": "oracle",
                 "sample": f"FP64 numpy oracle, same workload, {len(times)} step(s) timed at "
                           f"n={ref.n - len(times)}..{ref.n - 1} after {SATURATE} untimed steps from n=1",
                 "sec_per_step": per}


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores, same metric and workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload != WORKLOAD:
        print(json.dumps({"impl": "reference", "unavailable": "the FP64 oracle needs minutes per unit-cell step "
                          f"at {args.workload}; its timed arm runs on {WORKLOAD}"}), flush=True)
        return
    mpo, seed = make_workload(0)
    from oracle.idmrg import ParallelIDMRG
    ref = ParallelIDMRG.from_mpo(mpo, m=args.m)
    while ref.n <= SATURATE:
        ref.step()
    for _ in range(args.warmup):
        ref.step()
    t = time.perf_counter()
    for _ in range(args.steps):
        ref.step()
    dt = time.perf_counter() - t
    v = args.steps / dt
    cores = len(os.sched_getaffinity(0))
    line = {"metric": METRIC, "value": v, "unit": "unit-cell steps/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "ell": 16, "m": args.m, "solves_per_step": 8, "seed": seed,
                       "regime": f"saturated (n > {SATURATE})"},
            "cpu_baseline": {"value": v, "unit": "unit-cell steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} timed oracle steps after {SATURATE}+{args.warmup} untimed"},
            "e2e": {"value": v, "unit": "unit-cell steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch(args, pkg, dev, local, world, rank, dist):
    """The 64 disorder realisations of uneven unit cells and m, stepped
    together (idmrg_batch_step: host threads, one stream per realisation).
    value = realisation unit-cell steps per second (64 per batch step), timed
    by the wall clock around each batch step with the device synchronised on
    both sides (the realisations' kernels run on 64 streams)."""
    import torch
    from workloads import disorder_batch
    work = disorder_batch(64)
    threads = max(1, min(16, len(os.sched_getaffinity(0))))
    ctxs = [pkg.Context(mpo.W, mpo.phys_charge, mpo.bond_charge, m=m, prec=args.prec, lanczos_maxit=160,
                        stream=torch.cuda.Stream()) for _, mpo, m in work]
    for _ in range(SATURATE + max(args.warmup, 3)):
        pkg.batch_step(ctxs, threads)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    launches0 = sum(c.launch_count() for c in ctxs)
    h2d0 = sum(c.transfer_bytes()[0] for c in ctxs)
    d2h0 = sum(c.transfer_bytes()[1] for c in ctxs)
    clocks = Clocks(local)
    if dist is not None and dist.is_initialized():
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    wall = 0.0
    reps = None
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        reps = pkg.batch_step(ctxs, threads)
        torch.cuda.synchronize()
        wall += time.perf_counter() - t
    clk = clocks.stop()
    t_wall = reduce_max([wall], dist, dev)[0]
    launches = sum(c.launch_count() for c in ctxs) - launches0
    h2d = (sum(c.transfer_bytes()[0] for c in ctxs) - h2d0) // args.steps
    d2h = (sum(c.transfer_bytes()[1] for c in ctxs) - d2h0) // args.steps
    if rank == 0:
        v = world * len(ctxs) * args.steps / t_wall
        line = {
            "metric": METRIC, "value": v, "unit": "realisation unit-cell steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_wall * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp64tc": "bf16-digits(f64)+f64"}.get(args.prec, f"{args.prec}+f64"),
            "data": "synthetic",
            "config": {"workload": "disorder64", "realisations": len(ctxs),
                       "ell": "8/12/16/24 by r mod 4", "m": "128/256/512 by (r div 4) mod 3",
                       "couplings": "J ~ U[0.2, 1.8], PCG64 seed 1000 + r", "host_threads": threads,
                       "streams": len(ctxs), "regime": f"n > {SATURATE + max(args.warmup, 3)}",
                       "kept_max": int(max(int(max(r["kept"])) for r in reps)),
                       "timing": "wall clock per batch step, device synchronised on both sides",
                       "l2": "flushed before every timed step (256 MiB write, outside the timing)"},
            "roofline": None, "gpu_launches": launches,
            "e2e": {"value": v, "unit": "realisation unit-cell steps/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "note": "the batch API call is the timed region"},
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    for c in ctxs:
        c.close()
    if world > 1:
        dist.destroy_process_group()


def timed_run(pkg, mpo, m: int, prec: str, steps: int, warmup: int, dev, flush, dist, with_clocks: bool, local: int):
    """Saturate, warm up, then two timed regions of `steps` unit-cell steps,
    each step bracketed by CUDA events on the context's stream with the L2
    flushed before it (outside the events): the first without per-class
    timers (the step time, e2e wall clock and clocks), the second with the
    per-class event timers on (kernel classes and rooflines)."""
    import torch
    ctx = pkg.Context(mpo.W, mpo.phys_charge, mpo.bond_charge, m=m, prec=prec)
    for _ in range(SATURATE):
        ctx.unit_cell_step()
    for _ in range(max(warmup, 3)):
        ctx.unit_cell_step()
    stream = ctx.stream

    def region(profiled: bool, clocks):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        launches0 = ctx.launch_count()
        h2d0, d2h0 = ctx.transfer_bytes()
        ctx.profile_enable(profiled)
        if dist is not None and dist.is_initialized():
            dist.barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        torch.cuda.nvtx.range_push("timed")
        wall, reports = [], []
        for k in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            t = time.perf_counter()
            ev[k][0].record(stream)
            reports.append(ctx.unit_cell_step())
            ev[k][1].record(stream)
            torch.cuda.synchronize()
            wall.append(time.perf_counter() - t)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        clk = clocks.stop() if clocks else None
        if dist is not None and dist.is_initialized():
            dist.barrier()
        out = {"step_ms": sum(a.elapsed_time(b) for a, b in ev), "wall_s": sum(wall), "reports": reports,
               "clocks": clk, "launches": ctx.launch_count() - launches0}
        h2d1, d2h1 = ctx.transfer_bytes()
        out["h2d"] = (h2d1 - h2d0) // steps
        out["d2h"] = (d2h1 - d2h0) // steps
        if profiled:
            out["prof"] = ctx.profile_read()
        ctx.profile_enable(False)
        return out

    res = region(False, Clocks(local) if with_clocks else None)
    prof = region(True, None)
    res["prof"] = prof["prof"]
    res["prof_step_ms"] = prof["step_ms"]
    res["ctx"] = ctx
    return res


def observables_leg(ctx, ell: int) -> dict:
    """Uniform-MPS observables of the final state (Eq. mps2), outside the timed
    steps: the l nearest-neighbour bond strengths (unit embedding, both fixed
    points by power iteration, environments, walks) and the transfer spectrum
    (correlation length), each timed on the wall clock around its API call."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    try:
        v = ctx.spin_dot([(i, i + 1) for i in range(ell)])
        t1w = time.perf_counter()
        t1, t2, xi, it, conv = ctx.transfer_spectrum()
        t2w = time.perf_counter()
    except Exception as e:  # reported, not fatal: the step measurement stands
        return {"error": str(e)}
    return {"bond_strengths_ms": (t1w - t0) * 1e3, "spectrum_ms": (t2w - t1w) * 1e3,
            "bond_strength_mean": float(sum(v) / len(v)), "bond_strength_min": float(min(v)),
            "bond_strength_max": float(max(v)), "t1": t1, "t2_abs": t2, "xi_unit_cells": xi,
            "spectrum_iterations": it, "spectrum_converged": conv}


def max_de_per_site(ra, rb):
    """Largest |e_a - e_b| / (2n+2) over the superblocks of steps with equal n."""
    worst = 0.0
    by_n = {int(r["n"]): r for r in rb}
    for r in ra:
        o = by_n.get(int(r["n"]))
        if o is None:
            continue
        sites = 2 * int(r["n"]) + 2
        for x, y in zip(r["energy"], o["energy"]):
            worst = max(worst, abs(float(x) - float(y)) / sites)
    return worst


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--prec", default="tf32x3", choices=["fp64", "tf32x3", "bf16x3", "fp64tc"])
    ap.add_argument("--m", type=int, default=None, help="kept states (default: the workload's m)")
    ap.add_argument("--workload", default=WORKLOAD, choices=[WORKLOAD, "yc4_j1j2_l8_m1024", "disorder64"],
                    help="random-bond chain l=16 m=256 (the metric's workload), the YC4 J1-J2 cylinder, "
                         "or 64 disorder realisations stepped together")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-observables", action="store_true")
    args = ap.parse_args()
    if args.m is None:
        args.m = 256 if args.workload == WORKLOAD else 1024
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    import paper_1606_06790_gb300 as pkg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.workload == "disorder64":
        return run_batch(args, pkg, dev, local, world, rank, dist)
    mpo, seed = make_workload(rank, args.workload)
    ell = len(mpo.W)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    run = timed_run(pkg, mpo, args.m, args.prec, args.steps, args.warmup, dev, flush, dist, True, local)
    cmp = None
    if args.prec != "fp64" and not args.no_fp64_compare:
        cmp = timed_run(pkg, mpo, args.m, "fp64", args.steps, args.warmup, dev, flush, dist, False, local)
    t_dev, t_wall = run["step_ms"] * 1e-3, run["wall_s"]
    t_dev64 = cmp["step_ms"] * 1e-3 if cmp else 0.0
    t_dev, t_wall, t_dev64 = reduce_max([t_dev, t_wall, t_dev64], dist, dev)
    pk = peaks()
    prof = run["prof"]
    dom = max(prof, key=lambda k: prof[k]["ms"])
    roof = class_roofline(dom, prof[dom], args.prec, pk)
    kernels = {k: {"ms_per_step": v["ms"] / args.steps, "launches_per_step": v["launches"] / args.steps,
                   "gflops_per_s": (v["flops"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else 0.0,
                   "gbytes_per_s": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else 0.0}
               for k, v in prof.items()}
    ctx = run["ctx"]
    flops, _ = ctx.heff_cost(-1)
    last = run["reports"][-1]
    if rank != 0:
        ctx.close()
        if cmp is not None:
            cmp["ctx"].close()
        if world > 1:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": job_value(world, args.steps, t_dev), "unit": "unit-cell steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_dev * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp64tc": "bf16-digits(f64)+f64"}.get(args.prec, f"{args.prec}+f64"),
        "data": "synthetic",
        "config": {"workload": args.workload, "ell": ell, "m": args.m, "solves_per_step": ell // 2, "seed": seed,
                   "regime": f"saturated (n > {SATURATE}, D = {int(max(last['kept']))})",
                   "precision": args.prec + ("" if args.prec == "fp64" else " H_eff psi; FP64 Lanczos and SVD"),
                   "fp64_restart_matvecs": "BF16 digit slices on the tensor cores (FP64-accurate)"
                   if args.prec in ("tf32x3", "bf16x3") else None,
                   "parallelism": f"{world} independent realisation(s), one per GPU",
                   "l2": "flushed before every timed step (256 MiB write, outside the events)"},
        "roofline": roof,
        "roofline_heff": heff_roofline(prof, args.prec, pk),
        "gpu_launches": run["launches"],
        "e2e": {"value": job_value(world, args.steps, t_wall), "unit": "unit-cell steps/s",
                "h2d_bytes_per_step": run["h2d"], "d2h_bytes_per_step": run["d2h"],
                "note": "wall clock around idmrg_unit_cell_step: host block tables in, step report out"},
        "kernels": kernels,
        "kernels_note": ("per-class CUDA-event timers of a second timed region of the same length "
                         f"({run['prof_step_ms'] / args.steps:.2f} ms per step with the timers on)"),
        "svd": ctx.svd_stats(),
        "heff": {"flops_per_matvec_all_superblocks": flops,
                 "lanczos_iters_last_step": [int(x) for x in last["iters"]]},
        "clocks": run["clocks"],
        "energy_per_site_last": float(last["energy"][0] / (2 * last["n"] + 2)),
    }
    if not args.no_observables:
        line["observables"] = observables_leg(ctx, ell)
    if cmp is not None:
        line["fp64"] = {"value": job_value(world, args.steps, t_dev64), "unit": "unit-cell steps/s",
                        "ms_per_step": t_dev64 * 1e3 / args.steps,
                        "max_abs_de_per_site": max_de_per_site(run["reports"], cmp["reports"]),
                        "heff_roofline": heff_roofline(cmp["prof"], "fp64", pk)}
        cmp["ctx"].close()
    if world == 1 and not args.no_cpu_baseline and args.workload == WORKLOAD:
        _, cb = cpu_baseline(mpo, args.m)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
    print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
