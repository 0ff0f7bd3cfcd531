#!/usr/bin/env python
"""Parallel-iDMRG benchmark on GB300: unit-cell steps per second.

A step is one parallel iteration n (Sec. 3): the l/2 two-site superblocks
of the unit cell are solved (Lanczos on H_eff psi), truncated by SVD and
renormalised, all through the C ABI of libidmrg.  Workload: S=1/2 random-bond
Heisenberg chain, l = 16 (8 superblocks per step), J_k ~ U[0.5, 1.5] from
PCG64 seed 1606, m = 256, measured in the saturated regime (D = m).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp64] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun each rank runs its own
disorder realisation (seed 1606 + rank): independent problems, no exchange.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
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
HBM_FALLBACK, BF16_FALLBACK = 6800.0, 1900.0
FP64_ALU_PEAK = 152 * 2070e6 * 4 / 1e9   # GFLOP/s: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p["hbm_gbs"], p["bf16_tflops"], p.get("bf16_tflops_sustained", p["bf16_tflops"]), "measured"
    except Exception:
        return HBM_FALLBACK, BF16_FALLBACK, 1700.0, "fallback"


def make_workload(rank: int, m: int):
    from workloads import build_mpo, random_chain_bonds
    seed = 1606 + rank
    return build_mpo(random_chain_bonds(16, 0.5, 1.5, seed), 16), seed


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


KERNEL_SOURCES = {"heff_gemm": ["kernels_f64.cu"], "lanczos_vec": ["kernels_lanczos.cu"],
                  "svd": ["kernels_svd.cu"], "env": ["kernels_f64.cu"], "heff_wstage": ["kernels_f64.cu"]}


def traffic_for(kclass: str):
    """DRAM bytes per launch from a committed ncu summary, if the kernel is unchanged since."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        e = t[kclass]
        if e.get("source_hash") == source_hash(*KERNEL_SOURCES[kclass]):
            return e["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


def roofline(prof: dict, prec: str, hbm: float, bf16: float, src: str):
    dom = max(prof, key=lambda k: prof[k]["ms"])
    d = prof[dom]
    sec = d["ms"] * 1e-3
    per_launch_ms = d["ms"] / max(d["launches"], 1)
    if dom in ("heff_gemm", "env", "heff_wstage", "predict") and d["flops"] > 0:
        if prec == "fp64":
            achieved = d["flops"] / sec / 1e9
            return dom, {"bound": "alu", "achieved": achieved, "peak": FP64_ALU_PEAK, "unit": "GFLOP/s",
                         "frac": achieved / FP64_ALU_PEAK, "traffic": traffic_for(dom),
                         "kernel": dom, "launch_ms": per_launch_ms,
                         "peak_source": "FP64 FMA units x clock (152 SMs x 2 FMA/clk x 2.07 GHz)"}
        peak = bf16 * (1.1 / 2.25) if prec == "tf32x3" else bf16
        achieved = d["flops"] / sec / 1e12
        return dom, {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic_for(dom), "kernel": dom,
                     "launch_ms": per_launch_ms, "peak_source": f"{src} bf16 x nominal tf32/bf16 ratio"}
    achieved = d["bytes"] / sec / 1e9 if d["bytes"] > 0 else 0.0
    return dom, {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                 "traffic": traffic_for(dom), "kernel": dom, "launch_ms": per_launch_ms,
                 "peak_source": f"{src} copy bandwidth"}


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
    mpo, seed = make_workload(0, args.m)
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--prec", default="fp64", choices=["fp64", "tf32x3", "bf16x3"])
    ap.add_argument("--m", type=int, default=256)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    import paper_1606_06790_gb300 as pkg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mpo, seed = make_workload(rank, args.m)
    ctx = pkg.Context(mpo.W, mpo.phys_charge, mpo.bond_charge, m=args.m, prec=args.prec)
    for _ in range(SATURATE):
        ctx.unit_cell_step()
    for _ in range(max(args.warmup, 3)):
        ctx.unit_cell_step()
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = ctx.stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = Clocks(local)
    launches0 = ctx.launch_count()
    h2d0, d2h0 = ctx.transfer_bytes()
    ctx.profile_enable(True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    torch.cuda.nvtx.range_push("timed")
    wall = []
    reports = []
    for k in range(args.steps):
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
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    step_ms = sum(a.elapsed_time(b) for a, b in ev)
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    launches = ctx.launch_count() - launches0
    h2d1, d2h1 = ctx.transfer_bytes()
    t_dev = step_ms * 1e-3
    t_wall = sum(wall)
    if world > 1:
        tt = torch.tensor([t_dev, t_wall], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_dev, t_wall = float(tt[0]), float(tt[1])
    value = world * args.steps / t_dev
    e2e = world * args.steps / t_wall
    hbm, bf16, bf16s, src = peaks()
    dom, roof = roofline(prof, args.prec, hbm, bf16, src)
    kernels = {k: {"ms_per_step": v["ms"] / args.steps, "launches_per_step": v["launches"] / args.steps,
                   "gflops_per_s": (v["flops"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else 0.0,
                   "gbytes_per_s": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else 0.0}
               for k, v in prof.items()}
    flops, _ = ctx.heff_cost(-1)
    last = reports[-1]
    if rank != 0:
        ctx.close()
        if world > 1:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": "unit-cell steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.prec == "fp64" else args.prec, "data": "synthetic",
        "config": {"workload": WORKLOAD, "ell": 16, "m": args.m, "solves_per_step": 8, "seed": seed,
                   "regime": f"saturated (n > {SATURATE}, D = {int(max(last['kept']))})",
                   "precision": args.prec, "parallelism": f"{world} independent realisation(s)",
                   "l2": "flushed before every timed step (256 MiB write, outside the events)"},
        "roofline": roof,
        "gpu_launches": launches,
        "e2e": {"value": e2e, "unit": "unit-cell steps/s",
                "h2d_bytes_per_step": (h2d1 - h2d0) // args.steps, "d2h_bytes_per_step": (d2h1 - d2h0) // args.steps,
                "note": "wall clock around idmrg_unit_cell_step with its host-side block tables and report"},
        "kernels": kernels,
        "svd": ctx.svd_stats(),
        "heff": {"flops_per_matvec_all_superblocks": flops,
                 "lanczos_iters_last_step": [int(x) for x in last["iters"]]},
        "clocks": clk,
        "energy_per_site_last": float(last["energy"][0] / (2 * last["n"] + 2)),
    }
    if world == 1 and not args.no_cpu_baseline:
        _, cb = cpu_baseline(mpo, args.m)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
    print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
