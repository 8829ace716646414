"""Writes tgv128_clip_oracle.json: the FP64 oracle's E_k / u0^2 and
Z / (u0/L)^2 trajectories of the periodic D3Q27 Taylor-Green vortex at
N = 128, Re = 1600, Ma = 0.2 with resolved BGK and with KC-MP (C_nu = 0.035),
sampled every 20 steps over t u0/L in [0, 20] (Sec. 7.1: at N = 128 the
kinetic-energy curves of the closures and of BGK are nearly indistinguishable,
the rate limiter clipping the SGS relaxation).  Calls only the oracle and the
seeded input generator; about 80 minutes on 8 cores.

    python tests/golden/make_tgv128_clip.py
"""
import json
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2605_19796_gb300 import inputs  # noqa: E402

N, RE, MA, EVERY, T_END = 128, 1600.0, 0.2, 20, 20.0
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
    t, ek, z = [], [], []
    step = 0
    while step <= T_END * T and (steps_max is None or step <= steps_max):
        d = oracle.diagnostics(f)
        t.append(step / T)
        ek.append(d[4] / u0 ** 2)
        z.append(d[5] / (u0 / L) ** 2)
        f = oracle.run(f, EVERY, closure=closure, nu=nu, c_nu=c_nu)
        step += EVERY
    return {"t": t, "ek": ek, "z": z}


if __name__ == "__main__":
    oracle.build()
    out = {"about": "oracle trajectories of the N = 128 Taylor-Green runs; written by make_tgv128_clip.py",
           "every_steps": EVERY}
    for name, closure, c_nu in RUNS:
        out[name] = trajectory(closure, c_nu)
        print(name, "done", flush=True)
    with open(os.path.join(HERE, "tgv128_clip_oracle.json"), "w") as fp:
        json.dump(out, fp)
