"""Storage-precision study: FP32 vs weight-shifted FP16 / BF16 population storage.

Runs the same decaying-turbulence case (D3Q27, KC-MP, seeded HIT) with every
storage format and reports, against the FP64-storage run of the same case (the
FP64 path is parity-checked against the CPU oracle to 1e-12), per field:
max and rms error of rho and u, relative error of the kinetic energy, and the
relative L2 error of the energy spectrum E(k); plus MLUPS of each storage.
Weight-shifted storage keeps g_i = f_i - w_i (FP32 arithmetic in the kernel),
which puts the 10-bit (FP16) or 7-bit (BF16) mantissa on the small deviation
from the lattice weights instead of on f_i itself.
"""
from __future__ import annotations

import time
from typing import Dict, Sequence

import torch

from . import inputs, lbm
from .learned import spectrum


def _fields(s: lbm.Solver):
    nx, ny, nz = s.shape
    r = torch.empty((nz, ny, nx), dtype=torch.float64, device="cuda")
    u = torch.empty((3, nz, ny, nx), dtype=torch.float64, device="cuda")
    s.moments_device(r, u)
    torch.cuda.synchronize()
    return r, u


def run(n: int = 64, steps: int = 200, nu: float = 1e-4, k0: float = 4.0, urms: float = 0.04, seed: int = 0,
        storages: Sequence[str] = ("fp64", "fp32", "fp16", "bf16"), closure: str = "kcmp") -> Dict:
    rho0, u0 = inputs.hit_fields(n, k0=k0, urms=urms, seed=seed, device="cuda")
    res = {}
    ref = None
    for st in storages:
        with lbm.Solver(27, (n, n, n), nu, closure=closure, storage=st) as s:
            s.init_velocity_device(rho0, u0)
            s.step(2)
            s.synchronize()
            t0 = time.perf_counter()
            s.step(steps - 2)
            s.synchronize()
            dt = time.perf_counter() - t0
            r, u = _fields(s)
        e = spectrum(u)
        ek = float(0.5 * (r * (u ** 2).sum(0)).mean())
        res[st] = {"mlups": n ** 3 * (steps - 2) / dt / 1e6, "E_k": ek}
        if ref is None:
            ref = (r, u, e, ek)
            continue
        rr, ur, er, ekr = ref
        kmax = n // 2
        res[st].update({
            "rho_max_err": float((r - rr).abs().max()), "rho_rms_err": float(((r - rr) ** 2).mean().sqrt()),
            "u_max_err": float((u - ur).abs().max()), "u_rms_err": float(((u - ur) ** 2).mean().sqrt()),
            "E_k_rel_err": abs(ek - ekr) / ekr,
            "spectrum_rel_l2": float(torch.sqrt(((e[1:kmax] - er[1:kmax]) ** 2).sum() / (er[1:kmax] ** 2).sum())),
        })
    return res


def main(argv=None) -> Dict:
    """Storage-precision study of one decaying-turbulence case; prints one JSON line."""
    import argparse
    import json

    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--closure", default="kcmp")
    a = ap.parse_args(argv)
    res = run(n=a.n, steps=a.steps, closure=a.closure)
    print(json.dumps({"n": a.n, "steps": a.steps, "closure": a.closure, "results": res}), flush=True)
    return res


if __name__ == "__main__":
    main()
