"""Writes kcrb_sensitivity_tgv64_oracle.json: the FP64 oracle's E_k / u0^2 and
Z / (u0/L)^2 trajectories of the App. G comparison (KC-RB raw against Hermite,
and KC-RR as the Hermite-consistent reference; periodic D3Q27 TGV, N = 64,
Re = 1600, Ma = 0.2, C_nu = 0.02), sampled every 10 steps over t u0/L in
[0, 20].  Calls only the oracle and the seeded input generator; takes about
eight minutes on 8 cores.

    python tests/golden/make_kcrb_sensitivity.py
"""
import json
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2605_19796_gb300 import inputs  # noqa: E402

N, RE, MA, C_NU, EVERY, T_END = 64, 1600.0, 0.2, 0.02, 10, 20.0


def case():
    """u0, L_TGV, nu, the time unit L_TGV / u0 in steps, and the initial fields."""
    u0 = MA * math.sqrt(oracle.THETA)
    L = N / (2 * math.pi)
    rho, u = inputs.tgv_fields(N, u0=u0)
    return u0, L, u0 * L / RE, L / u0, rho, u


def trajectory(closure, steps_max=None):
    u0, L, nu, T, rho, u = case()
    f = oracle.init_equilibrium(27, rho, u)
    t, ek, z = [], [], []
    step = 0
    while step <= T_END * T and (steps_max is None or step <= steps_max):
        d = oracle.diagnostics(f)
        t.append(step / T)
        ek.append(d[4] / u0 ** 2)
        z.append(d[5] / (u0 / L) ** 2)
        f = oracle.run(f, EVERY, closure=closure, nu=nu, c_nu=C_NU)
        step += EVERY
    return {"t": t, "ek": ek, "z": z}


if __name__ == "__main__":
    oracle.build()
    out = {"about": "oracle trajectories of the App. G comparison; written by make_kcrb_sensitivity.py",
           "every_steps": EVERY, "hermite": trajectory(2), "raw": trajectory(3), "kcrr": trajectory(4)}
    with open(os.path.join(HERE, "kcrb_sensitivity_tgv64_oracle.json"), "w") as fp:
        json.dump(out, fp)
