#!/usr/bin/env python
"""Benchmark of the fused kinetic-closure LES step on GB300.

Metric: MLUPS (million lattice-cell updates per second) of the fused
stream-and-collide step, with its fraction of the HBM roofline.  Default
workload: decaying homogeneous isotropic turbulence, periodic 512^3, D3Q27,
FP32 storage and arithmetic, KC-MP closure (C_nu = 0.035), nu = 1e-4
(k0 = 4, u_rms = 0.04).  One "step" is one time step of the whole lattice (one
launch of the fused kernel).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Prints ONE JSON line on stdout (rank 0); progress goes to stderr.
Multi-GPU (torchrun): every rank advances its own replica box (independent
problems, no collective in the data path, weak scaling); rank 0 reports the
aggregate.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "hit512_d3q27_fp32_kcmp": dict(n=512, q=27, storage="fp32", closure="kcmp", nu=1e-4, k0=4.0, urms=0.04),
    "hit256_d3q27_fp32_kcmp": dict(n=256, q=27, storage="fp32", closure="kcmp", nu=1e-4, k0=4.0, urms=0.04),
    "hit512_d3q27_fp16_kcmp": dict(n=512, q=27, storage="fp16", closure="kcmp", nu=1e-4, k0=4.0, urms=0.04),
    "hit512_d3q27_bf16_kcmp": dict(n=512, q=27, storage="bf16", closure="kcmp", nu=1e-4, k0=4.0, urms=0.04),
    "hit512_d3q19_fp32_kcmp": dict(n=512, q=19, storage="fp32", closure="kcmp", nu=1e-4, k0=4.0, urms=0.04),
    "hit512_d3q27_fp32_bgk": dict(n=512, q=27, storage="fp32", closure="bgk", nu=1e-4, k0=4.0, urms=0.04),
}
DEFAULT_WORKLOAD = "hit512_d3q27_fp32_kcmp"
ELEM = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}
DTYPE = {"fp64": "f64", "fp32": "f32", "fp16": "f32 (f16 storage)", "bf16": "f32 (bf16 storage)"}
METRIC = "MLUPS (fused KC-LES stream-collide step)"
FALLBACK_HBM_GBS = 6800.0
# the oracle sample that stands in for the workload on the host cores
CPU_SAMPLE_N = 64


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in ("lbm_step.cuh", "lbm_step_inst.cuh", "lbm_lattice.cuh"):
        with open(os.path.join(ROOT, "paper_2605_19796_gb300", "csrc", f), "rb") as fp:
            h.update(fp.read())
    return h.hexdigest()[:16]


def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fp:
            return float(json.load(fp)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def traffic_per_cell(workload: str):
    """DRAM bytes per cell update of the step kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    try:
        with open(p) as fp:
            d = json.load(fp)
        e = d.get(workload)
        if e and e.get("kernel_hash") == kernel_hash():
            return float(e["dram_bytes_per_cell"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fp = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fp.close()
        rows = []
        with open(self.path) as fp:
            for line in fp:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def cpu_baseline(wl: dict, budget_s: float = 15.0, steps: int = 0):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample of
    the workload: a 64^3 box of the same turbulence recipe, lattice and closure."""
    import oracle
    from paper_2605_19796_gb300 import inputs

    oracle.build()
    n = CPU_SAMPLE_N
    rho, u = inputs.hit_fields(n, k0=wl["k0"], urms=wl["urms"], seed=0)
    f = oracle.init_equilibrium(wl["q"], rho, u)
    cl = {"bgk": 0, "kcmp": 1, "kcrb_hermite": 2, "kcrb_raw": 3}[wl["closure"]]
    cnu = {"bgk": 0.0, "kcmp": 0.035, "kcrb_hermite": 0.02, "kcrb_raw": 0.02}[wl["closure"]]
    t = time.perf_counter()
    f = oracle.run(f, 1, closure=cl, nu=wl["nu"], c_nu=cnu)
    t1 = time.perf_counter() - t
    k = steps or max(1, min(200, int(budget_s / max(t1, 1e-6))))
    t = time.perf_counter()
    oracle.run(f, k, closure=cl, nu=wl["nu"], c_nu=cnu)
    dt = time.perf_counter() - t
    return {"value": n ** 3 * k / dt / 1e6, "unit": "MLUPS", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{n}^3 box of the same recipe (D3Q{wl['q']}, {wl['closure']}, FP64 oracle), {k} steps, "
                      f"{dt:.1f} s"}


def run_reference(args, wl, rank):
    """Reference arm: the FP64 oracle on the host cores (rank 0 only)."""
    if rank != 0:
        return
    import oracle
    from paper_2605_19796_gb300 import inputs

    oracle.build()
    n = CPU_SAMPLE_N
    rho, u = inputs.hit_fields(n, k0=wl["k0"], urms=wl["urms"], seed=0)
    f = oracle.init_equilibrium(wl["q"], rho, u)
    cl = {"bgk": 0, "kcmp": 1, "kcrb_hermite": 2, "kcrb_raw": 3}[wl["closure"]]
    cnu = {"bgk": 0.0, "kcmp": 0.035, "kcrb_hermite": 0.02, "kcrb_raw": 0.02}[wl["closure"]]
    f = oracle.run(f, args.warmup, closure=cl, nu=wl["nu"], c_nu=cnu)
    t = time.perf_counter()
    oracle.run(f, args.steps, closure=cl, nu=wl["nu"], c_nu=cnu)
    dt = time.perf_counter() - t
    v = n ** 3 * args.steps / dt / 1e6
    out = {"metric": METRIC, "value": v, "unit": "MLUPS", "impl": "reference", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "sample": f"{n}^3 box of the same recipe on the host cores"},
           "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": oracle.num_threads(), "kind": "oracle",
                            "sample": f"{n}^3 D3Q{wl['q']} {wl['closure']} FP64, {args.steps} steps"},
           "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--tile-y", type=int, default=0)
    ap.add_argument("--zchunk", type=int, default=0)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    wl = WORKLOADS[args.workload]

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, wl, rank)
        return

    import numpy as np
    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist

        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2605_19796_gb300 import build, inputs

    build.build()
    from paper_2605_19796_gb300 import lbm

    n, q = wl["n"], wl["q"]
    N = n ** 3
    stream = torch.cuda.Stream(device=dev)
    log(f"[bench] {args.workload}: {n}^3 D3Q{q} {wl['storage']} {wl['closure']} rank {rank}/{world}")
    rho_d, u_d = inputs.hit_fields(n, k0=wl["k0"], urms=wl["urms"], seed=rank, device=dev)
    torch.cuda.synchronize()
    s = lbm.Solver(q, (n, n, n), wl["nu"], closure=wl["closure"], storage=wl["storage"], stream=stream,
                   tile_y=args.tile_y, zchunk=args.zchunk)
    s.init_velocity_device(rho_d, u_d)
    s.step(args.warmup)
    s.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    launches0 = s.kernel_launches
    barrier()
    torch.cuda.synchronize()
    ev[0].record(stream)
    for k in range(args.steps):
        s.step(1)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    gpu_launches = s.kernel_launches - launches0
    s.synchronize()  # raises on a non-finite field
    t_ms = ev[0].elapsed_time(ev[-1])
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    t_max = t_ms
    if dist is not None:
        tt = torch.tensor([t_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
    value = N * args.steps * world / (t_max * 1e-3) / 1e6

    # roofline of the step kernel (one launch per step)
    kern_s = sum(per) / len(per) * 1e-3
    alg_bytes = 2 * q * ELEM[wl["storage"]] * N
    peak, peak_src = measured_peak_hbm()
    achieved = alg_bytes / kern_s / 1e9
    tpc = traffic_per_cell(args.workload)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": (tpc * N if tpc is not None else None), "peak_source": peak_src,
                "algorithmic_bytes_per_cell": 2 * q * ELEM[wl["storage"]], "frac_of_nominal_8TBs": achieved / 8000.0}

    # end to end through the C ABI with pinned host buffers:
    # lbm_init_velocity (H2D of rho, u) + K steps + lbm_moments (D2H of rho, u)
    e2e = None
    if not args.no_e2e:
        rho_h = torch.empty((n, n, n), dtype=torch.float64, pin_memory=True)
        u_h = torch.empty((3, n, n, n), dtype=torch.float64, pin_memory=True)
        rho_h.copy_(rho_d)
        u_h.copy_(u_d)
        del rho_d, u_d
        torch.cuda.synchronize()
        rho_o = torch.empty((n, n, n), dtype=torch.float64, pin_memory=True)
        u_o = torch.empty((3, n, n, n), dtype=torch.float64, pin_memory=True)
        barrier()
        t0 = time.perf_counter()
        lbm.lbm_init_velocity(s.h, rho_h.numpy(), u_h.numpy())
        s.step(args.steps)
        lbm.lbm_moments(s.h, rho_o.numpy(), u_o.numpy())
        t1 = time.perf_counter() - t0
        barrier()
        if dist is not None:
            tt = torch.tensor([t1], device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            t1 = float(tt.item())
        e2e = {"value": N * args.steps * world / t1 / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": 32 * N // args.steps, "d2h_bytes_per_step": 32 * N // args.steps,
               "what": "lbm_init_velocity(pinned host rho,u) + K x lbm_step + lbm_moments(pinned host rho,u)"}
    s.close()

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(wl)
    out = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[wl["storage"]], "data": "synthetic",
        "config": {"workload": args.workload, "lattice": f"D3Q{q}", "cells": N, "shape": [n, n, n],
                   "closure": wl["closure"], "storage": wl["storage"], "nu": wl["nu"], "k0": wl["k0"],
                   "u_rms": wl["urms"], "kernel_launches_per_step": 1,
                   "l2": "inputs larger than L2 (two %.1f GB population buffers)" % (q * ELEM[wl["storage"]] * N / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches, "clocks": clocks,
        "kernel_ms": {"mean": sum(per) / len(per), "min": min(per), "max": max(per)},
    }
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
