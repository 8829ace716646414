"""Writes tgv64_clip_oracle.json: the FP64 oracle's E_k / u0^2 trajectories of
the periodic D3Q27 Taylor-Green vortex at N = 64, Re = 1600, Ma = 0.2 with
resolved BGK and with KC-MP (C_nu = 0.035), sampled every 10 steps from t = 0
until resolved BGK turns non-finite or t u0/L = 12, the N = 64 counterpart of
tgv128_clip_oracle.json (Sec. 7.1 contrasts the two resolutions: at N = 128
the closures' kinetic energy is nearly indistinguishable from BGK because the
rate limiter clips the SGS relaxation).  Calls only the oracle and the seeded
input generator; about two minutes on 8 cores.

    python tests/golden/make_tgv64_clip.py
"""
import json
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2605_19796_gb300 import inputs  # noqa: E402

N, RE, MA, EVERY, T_END = 64, 1600.0, 0.2, 10, 12.0
RUNS = (("bgk", 0, 0.0), ("kcmp", 1, 0.035))


def case():
    """u0, L_TGV, nu, the time unit L_TGV / u0 in steps, and the initial fields."""
    u0 = MA * math.sqrt(oracle.THETA)
    L = N / (2 * math.pi)
    rho, u = inputs.tgv_fields(N, u0=u0)
    return u0, L, u0 * L / RE, L / u0, rho, u


def trajectory(closure, c_nu, steps_max=None):
    u0, L, nu, T, rho, u = case()
    f = oracle.init_equilibrium(27, rho, u)
    t, ek = [], []
    step = 0
    while step <= T_END * T and (steps_max is None or step <= steps_max):
        d = oracle.diagnostics(f)
        if d[6] > 0 or not np.isfinite(d[4]):
            break
        t.append(step / T)
        ek.append(d[4] / u0 ** 2)
        f = oracle.run(f, EVERY, closure=closure, nu=nu, c_nu=c_nu)
        step += EVERY
    return {"t": t, "ek": ek}


if __name__ == "__main__":
    oracle.build()
    out = {"about": "oracle trajectories of the N = 64 Taylor-Green runs; written by make_tgv64_clip.py",
           "every_steps": EVERY}
    for name, closure, c_nu in RUNS:
        out[name] = trajectory(closure, c_nu)
        print(name, "done", len(out[name]["t"]), out[name]["t"][-1], flush=True)
    with open(os.path.join(HERE, "tgv64_clip_oracle.json"), "w") as fp:
        json.dump(out, fp)
