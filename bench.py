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
import re
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
    "hit256_d3q27_fp16_kcmp": dict(n=256, q=27, storage="fp16", closure="kcmp", nu=1e-4, k0=4.0, urms=0.04),
    "hit256_d3q27_bf16_kcmp": dict(n=256, q=27, storage="bf16", closure="kcmp", nu=1e-4, k0=4.0, urms=0.04),
    "hit512_d3q19_fp32_kcmp": dict(n=512, q=19, storage="fp32", closure="kcmp", nu=1e-4, k0=4.0, urms=0.04),
    "hit256_d3q19_fp32_kcmp": dict(n=256, q=19, storage="fp32", closure="kcmp", nu=1e-4, k0=4.0, urms=0.04),
    "hit512_d3q19_fp16_kcmp": dict(n=512, q=19, storage="fp16", closure="kcmp", nu=1e-4, k0=4.0, urms=0.04),
    "hit512_d3q27_fp32_bgk": dict(n=512, q=27, storage="fp32", closure="bgk", nu=1e-4, k0=4.0, urms=0.04),
    "hit512_d3q27_fp32_kcrr": dict(n=512, q=27, storage="fp32", closure="kcrr", nu=1e-4, k0=4.0, urms=0.04),
    "hit256_d3q27_fp32_kcrr": dict(n=256, q=27, storage="fp32", closure="kcrr", nu=1e-4, k0=4.0, urms=0.04),
    "hit512_d3q27_fp32_kcrb_raw": dict(n=512, q=27, storage="fp32", closure="kcrb_raw", nu=1e-4, k0=4.0, urms=0.04),
    "hit256_d3q27_fp64_kcmp": dict(n=256, q=27, storage="fp64", closure="kcmp", nu=1e-4, k0=4.0, urms=0.04),
    "hit128_d3q27_fp64_kcmp": dict(n=128, q=27, storage="fp64", closure="kcmp", nu=1e-4, k0=4.0, urms=0.04),
    # learned closure (KC-MP with the network's m_sgs, fused BF16 tensor-core inference)
    "hit256_d3q27_fp32_learned": dict(n=256, q=27, storage="fp32", closure="learned", nu=2.5e-5, k0=4.0, urms=0.04),
    "hit128_d3q27_fp32_learned": dict(n=128, q=27, storage="fp32", closure="learned", nu=2.5e-5, k0=4.0, urms=0.04),
    "hit256_d3q27_fp32_kcmp_nu2.5e-5": dict(n=256, q=27, storage="fp32", closure="kcmp", nu=2.5e-5, k0=4.0,
                                            urms=0.04),
    # 64 independent periodic 64^3 boxes, per-box nu uniform in [5e-5, 5e-4], distinct seeds,
    # all steps of the timed region replayed as one CUDA graph
    "ens64x64_d3q27_fp32_kcmp": dict(n=64, nbatch=64, q=27, storage="fp32", closure="kcmp", nu="ensemble", k0=4.0,
                                     urms=0.04),
    # plane channel 512 x 256 x 256, walls in y (halfway bounce-back), Re_tau ~ 180:
    # u_tau = 0.004, h = 128, nu = u_tau h / 180, F_x = u_tau^2 / h
    "channel512x256x256_d3q27_fp32_kcmp": dict(shape=(512, 256, 256), q=27, storage="fp32", closure="kcmp",
                                               nu=0.004 * 128 / 180, force=(0.004 ** 2 / 128, 0.0, 0.0),
                                               u_bulk=0.063),
    "channel512x256x256_d3q19_fp32_kcmp": dict(shape=(512, 256, 256), q=19, storage="fp32", closure="kcmp",
                                               nu=0.004 * 128 / 180, force=(0.004 ** 2 / 128, 0.0, 0.0),
                                               u_bulk=0.063),
    # the same channel at half the size in every direction (h = 64, Re_tau ~ 90
    # at the same u_tau): a case small enough for multi-pass ncu captures
    "channel256x128x128_d3q27_fp32_kcmp": dict(shape=(256, 128, 128), q=27, storage="fp32", closure="kcmp",
                                               nu=0.004 * 64 / 90, force=(0.004 ** 2 / 64, 0.0, 0.0),
                                               u_bulk=0.063),
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


KERNEL_SOURCES = ("lbm_lattice.cuh", "lbm_mbarrier.cuh", "lbm_mlp_infer.cuh", "lbm_mlp_tc.cuh", "lbm_tmem.cuh",
                  "lbm_step.cuh", "lbm_step_split.cuh", "lbm_step_tc.cuh", "lbm_step_v4.cuh")


def _code_only(text: str) -> str:
    """Source text without comments and with whitespace collapsed, so that a
    comment edit does not count as a kernel change."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_hash() -> str:
    """Hash of the code (comments and layout ignored) of the files that hold the
    step kernels' device code (the units that only instantiate them, and the
    host code that picks the launch, are checked through the launch recorded
    beside each record)."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2605_19796_gb300", "csrc", f), encoding="utf-8") as fp:
            h.update(_code_only(fp.read()).encode())
    return h.hexdigest()[:16]


def fp64_ops_per_cell(workload: str, launch: dict):
    """FP64 instructions and flops per cell update of the step kernel (FP64
    storage) from the committed ncu counts, if taken on the current kernel
    source and the same kernel instantiation."""
    p = os.path.join(ROOT, "profiles", "step_kernel_fp64_ops.json")
    try:
        with open(p) as fp:
            e = json.load(fp).get(workload)
        same = all(e.get("launch", {}).get(k) == launch.get(k) for k in ("variant", "tile_y")) if e else False
        if e and same and e.get("kernel_hash") == kernel_hash():
            return float(e["fp64_instructions_per_cell"]), float(e["fp64_flops_per_cell"])
    except Exception:
        pass
    return None


def warp_instructions_per_cell(workload: str, launch: dict):
    """Warp instructions per cell update of the step kernel (16-bit storage)
    from the committed ncu counts, if taken on the current kernel source and
    the same kernel instantiation."""
    p = os.path.join(ROOT, "profiles", "step_kernel_issue.json")
    try:
        with open(p) as fp:
            e = json.load(fp).get(workload)
        same = all(e.get("launch", {}).get(k) == launch.get(k) for k in ("variant", "tile_y")) if e else False
        if e and same and e.get("kernel_hash") == kernel_hash():
            return float(e["warp_instructions_per_cell"]), float(e["dram_bytes_per_cell"])
    except Exception:
        pass
    return None


# SM instruction issue: 4 schedulers per SM, one warp instruction each per clock
ISSUE_PER_SM_CLK = 4

# GB300 FP64 pipe: the nominal 1.25 TFLOP/s is 2 FP64 instructions per SM per
# clock on 152 SMs at the 2070 MHz maximum clock
FP64_INSTR_PER_SM_CLK = 2
N_SM = 152


def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fp:
            return float(json.load(fp)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def traffic_per_cell(workload: str, launch: dict):
    """DRAM bytes per cell update of the step kernel from the committed ncu
    summary, if it was taken on the current kernel source and the same kernel
    instantiation (variant, tile height) as this run's launch."""
    p = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    try:
        with open(p) as fp:
            d = json.load(fp)
        e = d.get(workload)
        same = all(e.get("launch", {}).get(k) == launch.get(k) for k in ("variant", "tile_y")) if e else False
        if e and same and e.get("kernel_hash") == kernel_hash():
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


def learned_weights():
    """Trained network if a checkpoint was saved next to the package, else a
    seeded initialisation with unit statistics (timing does not depend on the values)."""
    import numpy as np

    path = os.path.join(ROOT, "paper_2605_19796_gb300", "data", "learned_closure.npz")
    if os.path.exists(path):
        d = np.load(path)
        return {"params": d["params"], "stats": d["stats"], "source": "trained checkpoint"}
    from paper_2605_19796_gb300 import learned

    stats = np.concatenate([np.zeros(10), np.full(10, 1e-3), np.zeros(6), np.full(6, 1e-4)]).astype(np.float32)
    return {"params": learned.init_params(0), "stats": stats, "source": "seeded initialisation"}


def oracle_sample(wl: dict):
    """The bounded host-side sample of a workload that the FP64 oracle runs:
    a 64^3 box of the same turbulence recipe (one box of an ensemble, at the
    middle of its viscosity range), or a 64 x 32 x 32 slice of the channel."""
    import oracle
    from paper_2605_19796_gb300 import inputs

    oracle.build()
    # the learned closure's CPU stand-in is the analytic KC-MP it extends
    cl = {"bgk": 0, "kcmp": 1, "kcrb_hermite": 2, "kcrb_raw": 3, "kcrr": 4, "learned": 1}[wl["closure"]]
    cnu = {"bgk": 0.0, "kcmp": 0.035, "kcrb_hermite": 0.02, "kcrb_raw": 0.02, "kcrr": 0.02,
           "learned": 0.035}[wl["closure"]]
    bc, F = (0, 0, 0), (0.0, 0.0, 0.0)
    if "u_bulk" in wl:
        shape = (CPU_SAMPLE_N, CPU_SAMPLE_N // 2, CPU_SAMPLE_N // 2)
        rho, u = inputs.channel_fields(*shape, wl["u_bulk"], seed=0)
        bc, F, nu = (0, 1, 0), wl["force"], wl["nu"]
        desc = f"{shape[0]}x{shape[1]}x{shape[2]} channel slice"
    else:
        shape = (CPU_SAMPLE_N,) * 3
        rho, u = inputs.hit_fields(CPU_SAMPLE_N, k0=wl["k0"], urms=wl["urms"], seed=0)
        nu = 2.75e-4 if isinstance(wl["nu"], str) else wl["nu"]
        desc = f"{CPU_SAMPLE_N}^3 box of the same recipe"
    f = oracle.init_equilibrium(wl["q"], rho, u)
    run = lambda f, k: oracle.run(f, k, closure=cl, nu=nu, c_nu=cnu, bc=bc, F=F)
    return f, run, shape[0] * shape[1] * shape[2], desc


def cpu_baseline(wl: dict, budget_s: float = 25.0, steps: int = 0, single_budget_s: float = 8.0):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample of
    the workload; then the same sample on one thread (single_thread)."""
    import oracle

    f, run, cells, desc = oracle_sample(wl)

    def timed(f, budget):
        t = time.perf_counter()
        f = run(f, 1)
        t1 = time.perf_counter() - t
        k = steps or max(1, min(5000, int(budget / max(t1, 1e-6))))
        t = time.perf_counter()
        run(f, k)
        return k, time.perf_counter() - t

    cores = oracle.num_threads()
    k, dt = timed(f, budget_s)
    out = {"value": cells * k / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
           "sample": f"{desc} (D3Q{wl['q']}, {wl['closure']}, FP64 oracle), {k} steps, {dt:.1f} s"}
    if single_budget_s > 0 and cores > 1:
        oracle.set_num_threads(1)
        try:
            k1, dt1 = timed(f, single_budget_s)
        finally:
            oracle.set_num_threads(cores)
        out["single_thread"] = {"value": cells * k1 / dt1 / 1e6, "unit": "MLUPS", "cores": 1,
                                "sample": f"the same sample, {k1} steps, {dt1:.1f} s"}
    return out


def run_reference(args, wl, rank):
    """Reference arm: the FP64 oracle on the host cores (rank 0 only)."""
    if rank != 0:
        return
    import oracle

    f, run, cells, desc = oracle_sample(wl)
    f = run(f, args.warmup)
    t = time.perf_counter()
    run(f, args.steps)
    dt = time.perf_counter() - t
    v = cells * args.steps / dt / 1e6
    out = {"metric": METRIC, "value": v, "unit": "MLUPS", "impl": "reference", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "sample": f"{desc} on the host cores"},
           "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": oracle.num_threads(), "kind": "oracle",
                            "sample": f"{desc}, D3Q{wl['q']} {wl['closure']} FP64, {args.steps} steps"},
           "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


FORMS = ("hit512_d3q27_fp16_kcmp", "hit512_d3q27_bf16_kcmp", "hit256_d3q27_fp32_learned")


def time_form(lbm, wl: dict, stream, steps: int, warmup: int, peak: float) -> dict:
    """CUDA-event MLUPS of one workload's step (the same K-step graph replay as
    the headline) and its fraction of the HBM roofline."""
    import torch

    from paper_2605_19796_gb300 import inputs

    n = wl["n"]
    rho_d, u_d = inputs.hit_fields(n, k0=wl["k0"], urms=wl["urms"], seed=0, device="cuda")
    torch.cuda.synchronize()
    with lbm.Solver(wl["q"], (n, n, n), wl["nu"], closure=wl["closure"], storage=wl["storage"],
                    stream=stream) as s:
        s.init_velocity_device(rho_d, u_d)
        del rho_d, u_d
        src = None
        if wl["closure"] == "learned":
            w = learned_weights()
            s.set_learned_closure(w["params"], w["stats"])
            src = w["source"]
        s.step(warmup)
        s.step(steps)  # graph capture outside the timed region
        s.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        s.step(steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        s.synchronize()
        t = ev0.elapsed_time(ev1) * 1e-3
        cells = n ** 3 * steps
        gbs = 2 * wl["q"] * ELEM[wl["storage"]] * cells / t / 1e9
        out = {"mlups": cells / t / 1e6, "ms_per_step": t / steps * 1e3, "hbm_gbs": gbs, "hbm_frac": gbs / peak,
               "algorithmic_bytes_per_cell": 2 * wl["q"] * ELEM[wl["storage"]], "launch": s.launch_config}
        if src:
            out["network"] = src
        return out


def measure_forms(lbm, stream, steps: int, warmup: int, peak: float) -> dict:
    """The 16-bit storage forms (512^3 KC-MP) and the learned closure (256^3)
    beside the FP32 headline, each with the error it carries, measured in the
    same run on the GPU:
      - 16-bit storage: against the FP64-storage run of the same library (whose
        every population matches the FP64 oracle to 1e-12 in the parity tests)
        on 64^3 HIT (k0 = 4, u_rms = 0.04, nu = 1e-4, KC-MP), 100 steps;
      - learned closure: a posteriori, 128^3 coarse LES for 150 coarse steps from
        the box-filtered state of a 512^3 KC-MP run at step 400 (held-out seed
        99), E(k) relative L2 error over shells 1 .. 63 against the filtered fine
        run, beside KC-MP's on the same case (C_nu = 0.035 for both)."""
    from paper_2605_19796_gb300 import learned, precision

    out = {}
    for name in FORMS:
        log(f"[bench] form {name}")
        out[name] = time_form(lbm, WORKLOADS[name], stream, steps, warmup, peak)
    # both studies run on torch's default stream (the solvers' legacy default stream)
    prec = precision.run(n=64, steps=100, storages=("fp64", "fp16", "bf16"))
    for st in ("fp16", "bf16"):
        out[f"hit512_d3q27_{st}_kcmp"]["error"] = {
            k: prec[st][k] for k in ("u_rms_err", "u_max_err", "rho_rms_err", "E_k_rel_err", "spectrum_rel_l2")}
        out[f"hit512_d3q27_{st}_kcmp"]["error"]["against"] = (
            "FP64-storage run, 64^3 HIT k0 = 4, u_rms = 0.04, nu = 1e-4, KC-MP, 100 steps")
    w = learned_weights()
    t0 = time.perf_counter()
    ap = learned.a_posteriori(w["params"], w["stats"], n_fine=512, factor=4, seed=99, t0=400, coarse_steps=150,
                              closures=("kcmp", "learned"))
    out["hit256_d3q27_fp32_learned"]["error"] = {
        "spectrum_rel_l2": ap["learned"]["spectrum_rel_l2"], "kcmp_spectrum_rel_l2": ap["kcmp"]["spectrum_rel_l2"],
        "dissipation": ap["learned"]["dissipation"], "kcmp_dissipation": ap["kcmp"]["dissipation"],
        "filtered_fine_dissipation": ap["filtered_fine"]["dissipation"],
        "against": "box-filtered 512^3 KC-MP run (factor 4), held-out seed 99, 150 coarse steps from fine step 400",
        "seconds": round(time.perf_counter() - t0, 1)}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the 16-bit storage and learned-closure lines of the default run")
    ap.add_argument("--tile-y", type=int, default=0)
    ap.add_argument("--zchunk", type=int, default=0)
    ap.add_argument("--variant", type=int, default=0)
    ap.add_argument("--autotune", type=int, default=0,
                    help="run the library autotuner before the warm-up (1/0); the default launch is the measured one")
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

    from paper_2605_19796_gb300.replicas import Replicas

    rep = Replicas("nccl")
    if world == 1:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2605_19796_gb300 import build, inputs

    build.build()
    from paper_2605_19796_gb300 import lbm

    q = wl["q"]
    shape = tuple(wl["shape"]) if "shape" in wl else (wl["n"],) * 3
    nb = wl.get("nbatch", 1)
    nx, ny, nz = shape
    N = nx * ny * nz * nb  # cells updated per step (all boxes)
    stream = torch.cuda.Stream(device=dev)
    log(f"[bench] {args.workload}: {shape} x {nb} D3Q{q} {wl['storage']} {wl['closure']} rank {rank}/{world}")
    bc = (0, 0, 0)
    force = wl.get("force", (0.0, 0.0, 0.0))
    if "u_bulk" in wl:  # channel
        bc = (0, 1, 0)
        rho_d, u_d = inputs.channel_fields(nx, ny, nz, wl["u_bulk"], seed=rep.seed(), device=dev)
        nu = wl["nu"]
    elif nb > 1:  # ensemble of boxes with their own seeds and viscosities
        parts = [inputs.hit_fields(nx, k0=wl["k0"], urms=wl["urms"], seed=rep.seed(b, nb), device=dev)
                 for b in range(nb)]
        rho_d = torch.stack([p[0] for p in parts])
        u_d = torch.stack([p[1] for p in parts], dim=1).contiguous()
        del parts
        nu = inputs.ensemble_viscosities(nb, seed=rank)
    else:
        rho_d, u_d = inputs.hit_fields(nx, k0=wl["k0"], urms=wl["urms"], seed=rep.seed(), device=dev)
        nu = wl["nu"]
    torch.cuda.synchronize()
    s = lbm.Solver(q, shape, nu, closure=wl["closure"], storage=wl["storage"], stream=stream, bc=bc, force=force,
                   nbatch=nb, tile_y=args.tile_y, zchunk=args.zchunk, variant=args.variant)
    s.init_velocity_device(rho_d, u_d)
    weights = None
    if wl["closure"] == "learned":
        weights = learned_weights()
        s.set_learned_closure(weights["params"], weights["stats"])
    tuned = None
    if args.autotune:
        tuned = s.autotune()
        log(f"[bench] autotuned launch: {tuned}")
    s.step(args.warmup)
    s.synchronize()

    barrier = rep.barrier
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = s.kernel_launches
    s.step(args.steps)  # captures the K-step graph outside the timed region
    s.synchronize()
    barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    s.step(args.steps)  # one CUDA-graph launch of K fused-step kernels
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    gpu_launches = s.kernel_launches - launches0 - args.steps
    s.synchronize()  # raises on a non-finite field
    t_ms = ev0.elapsed_time(ev1)
    per = [t_ms / args.steps]
    t_max = rep.max_over_ranks(t_ms)
    value = rep.whole_job_rate(N * args.steps, t_max * 1e-3) / 1e6

    # roofline of the step kernel (one launch per step, back to back in the graph)
    kern_s = sum(per) / len(per) * 1e-3
    alg_bytes = 2 * q * ELEM[wl["storage"]] * N
    peak, peak_src = measured_peak_hbm()
    achieved = alg_bytes / kern_s / 1e9
    tpc = traffic_per_cell(args.workload, s.launch_config)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": (tpc * N if tpc is not None else None), "peak_source": peak_src,
                "algorithmic_bytes_per_cell": 2 * q * ELEM[wl["storage"]], "frac_of_nominal_8TBs": achieved / 8000.0}
    wi = warp_instructions_per_cell(args.workload, s.launch_config) if wl["storage"] in ("fp16", "bf16") else None
    if wi is not None:
        # 16-bit storage halves the bytes; the same FP32 arithmetic then bounds
        # the step by instruction issue
        ipeak = ISSUE_PER_SM_CLK * N_SM * 2070.0 * 1e6 / 1e9
        iach = wi[0] * N / kern_s / 1e9
        roofline = {"bound": "alu", "achieved": iach, "peak": ipeak, "unit": "G warp instructions/s",
                    "frac": iach / ipeak, "traffic": wi[1] * N,
                    "peak_source": "instruction issue: 4 schedulers per SM, one warp instruction each per clock, "
                                   "152 SMs at 2070 MHz",
                    "warp_instructions_per_cell": wi[0], "hbm_frac": achieved / peak,
                    "algorithmic_bytes_per_cell": 2 * q * ELEM[wl["storage"]]}
    ops = fp64_ops_per_cell(args.workload, s.launch_config) if wl["storage"] == "fp64" else None
    if ops is not None:
        # FP64 storage runs FP64 arithmetic, bound by GB300's FP64 pipe
        sm_mhz = 2070.0
        fpeak = FP64_INSTR_PER_SM_CLK * N_SM * sm_mhz * 1e6 / 1e9
        fach = ops[0] * N / kern_s / 1e9
        roofline = {"bound": "alu", "achieved": fach, "peak": fpeak, "unit": "G FP64 instructions/s",
                    "frac": fach / fpeak, "traffic": None,
                    "peak_source": "nominal FP64 rate 1.25 TFLOP/s = 2 FP64 instructions per SM per clock, "
                                   "152 SMs at 2070 MHz",
                    "fp64_instructions_per_cell": ops[0], "fp64_tflops": ops[1] * N / kern_s / 1e12,
                    "hbm_frac": achieved / peak}

    # end to end through the C ABI with pinned host buffers:
    # lbm_init_velocity (H2D of rho, u) + K steps + lbm_moments (D2H of rho, u).
    # FP32 and 16-bit storage take the FP32 host fields (lbm_init_velocity_f32 /
    # lbm_moments_f32: the equilibrium and the moments are FP32 arithmetic on
    # the device either way); FP64 storage the FP64 ones.  Both are listed.
    e2e = None
    if not args.no_e2e:
        def e2e_runs(dt):
            # page-locked host buffers from the library (lbm_host_alloc)
            rho_h = lbm.host_empty(tuple(rho_d.shape), dt)
            u_h = lbm.host_empty(tuple(u_d.shape), dt)
            torch.from_numpy(rho_h).copy_(rho_d)
            torch.from_numpy(u_h).copy_(u_d)
            torch.cuda.synchronize()
            rho_o = lbm.host_empty(rho_h.shape, dt)
            u_o = lbm.host_empty(u_h.shape, dt)
            init = lbm.lbm_init_velocity_f32 if dt == np.float32 else lbm.lbm_init_velocity
            mom = lbm.lbm_moments_f32 if dt == np.float32 else lbm.lbm_moments
            # three runs, each the whole path (upload, K steps, download); the
            # median is reported and every run listed (a single run now and then
            # meets a host-side stall of a few hundred ms in the copies)
            runs, phases = [], []
            for _ in range(3):
                barrier()
                t0 = time.perf_counter()
                init(s.h, rho_h, u_h)
                ta = time.perf_counter()
                s.step(args.steps)
                s.synchronize()
                tb = time.perf_counter()
                mom(s.h, rho_o, u_o)
                t1 = time.perf_counter() - t0
                barrier()
                runs.append(rep.whole_job_rate(N * args.steps, rep.max_over_ranks(t1)) / 1e6)
                phases.append([round(1e3 * (ta - t0), 1), round(1e3 * (tb - ta), 1), round(1e3 * (t0 + t1 - tb), 1)])
            nb_step = 4 * np.dtype(dt).itemsize * N // args.steps
            return {"value": sorted(runs)[1], "runs": runs, "phases_ms_init_steps_moments": phases,
                    "h2d_bytes_per_step": nb_step, "d2h_bytes_per_step": nb_step}

        f64 = e2e_runs(np.float64)
        if wl["storage"] == "fp64":
            e2e = dict(f64, unit="MLUPS", host_fields="f64",
                       what="median of 3 runs of lbm_init_velocity(host rho,u from lbm_host_alloc) + K x lbm_step + "
                            "lbm_moments(host rho,u from lbm_host_alloc)")
        else:
            f32 = e2e_runs(np.float32)
            e2e = dict(f32, unit="MLUPS", host_fields="f32", f64_fields=f64,
                       what="median of 3 runs of lbm_init_velocity_f32(host FP32 rho,u from lbm_host_alloc) + "
                            "K x lbm_step + lbm_moments_f32(host FP32 rho,u from lbm_host_alloc); f64_fields: "
                            "the same with lbm_init_velocity / lbm_moments and FP64 fields")
        del rho_d, u_d
    s_cfg = s.launch_config
    s.close()

    if not rep.root:
        rep.close()
        return
    forms = None
    if not args.no_forms and world == 1 and args.workload == DEFAULT_WORKLOAD:
        forms = measure_forms(lbm, stream, args.steps, args.warmup, peak)
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(wl)
    out = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[wl["storage"]], "data": "synthetic",
        "config": {"workload": args.workload, "lattice": f"D3Q{q}", "cells": N, "shape": list(shape), "boxes": nb,
                   "closure": wl["closure"], "storage": wl["storage"],
                   "nu": wl["nu"] if not isinstance(wl["nu"], str) else "uniform [5e-5, 5e-4] per box",
                   "kernel_launches_per_step": 1, "launch": s_cfg, "cuda_graph": "K steps replayed as one graph launch",
                   "l2": "inputs larger than L2 (two %.1f GB population buffers)" % (q * ELEM[wl["storage"]] * N / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches, "clocks": clocks,
        "kernel_ms": {"mean": sum(per) / len(per)},
    }
    if forms is not None:
        out["forms"] = forms
    print(json.dumps(out), flush=True)
    rep.close()


if __name__ == "__main__":
    main()
