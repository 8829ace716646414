"""The App. G comparison on the GPU: the library's FP64 path runs both KC-RB
reconstructions and KC-RR on the 64^3 Taylor-Green vortex over the paper's
window and must reproduce the printed maximum relative differences
(tests/golden/), and follow the oracle's stored trajectories of the same
runs."""
import json
import math
import os

import numpy as np
import pytest

from paper_2605_19796_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def lbm():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2605_19796_gb300 import build

    build.build()
    from paper_2605_19796_gb300 import lbm as _lbm

    return _lbm


def _gold():
    gold = {}
    with open(os.path.join(GOLDEN, "kcrb_sensitivity_tgv64.txt")) as fp:
        for line in fp:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split()
                gold[k] = float(v)
    return gold


def _runs(lbm, names):
    """E_k / u0^2 and Z / (u0/L)^2 of the App. G runs on the GPU's FP64 path,
    every 10 steps over t u0/L in [0, 20], each checked against the oracle's
    stored trajectory: 1e-9 relative up to t = 5, 1e-4 to the end (FP64
    rounding-order differences grow over the 1770 steps of a turbulent run
    but stay far below the closures' own differences)."""
    with open(os.path.join(GOLDEN, "kcrb_sensitivity_tgv64_oracle.json")) as fp:
        stored = json.load(fp)
    n, ma, re_, c_nu, every = 64, 0.2, 1600.0, 0.02, stored["every_steps"]
    u0 = ma * math.sqrt(1.0 / 3.0)
    L = n / (2 * math.pi)
    nu = u0 * L / re_
    T = L / u0
    rho, u = inputs.tgv_fields(n, u0=u0)
    traj = {}
    for name in names:
        ek, z = [], []
        closure = "kcrr" if name == "kcrr" else "kcrb_" + name
        with lbm.Solver(27, (n, n, n), nu, closure=closure, c_nu=c_nu, storage="fp64") as s:
            s.init_velocity(rho, u)
            step = 0
            while step <= 20.0 * T:
                d = s.diagnostics()
                ek.append(d[4] / u0 ** 2)
                z.append(d[5] / (u0 / L) ** 2)
                s.step(every)
                step += every
        traj[name] = {"ek": np.array(ek), "z": np.array(z)}
        t = np.array(stored[name]["t"])
        assert len(ek) == len(t)
        for key in ("ek", "z"):
            ref = np.array(stored[name][key])
            err = np.abs(traj[name][key] - ref) / np.abs(ref)
            assert err[t <= 5.0].max() <= 1e-9, (name, key, err[t <= 5.0].max())
            assert err.max() <= 1e-4, (name, key, err.max())
    return traj


def test_kcrb_sensitivity_tgv64_matches_app_g(lbm):
    """Periodic D3Q27 TGV, N = 64, Re = 1600, Ma = 0.2, C_nu = 0.02, FP64
    storage (App. G): the maximum relative differences between KC-RB raw
    and Hermite must match the printed 3.06 % and 12.82 % (2 % and 3 % of
    those values, as for the oracle), both differences changing sign, and
    every sample must follow the oracle's stored trajectory."""
    gold = _gold()
    traj = _runs(lbm, ("hermite", "raw"))
    for key, printed, tol in (("ek", gold["ek_max_rel_diff_percent"], 0.02),
                              ("z", gold["z_max_rel_diff_percent"], 0.03)):
        h, r = traj["hermite"][key], traj["raw"][key]
        d = r - h
        got = 100 * float(np.max(np.abs(d) / np.abs(h)))
        assert got == pytest.approx(printed, rel=tol), (key, got)
        assert (d > 0).any() and (d < 0).any()


def test_kcrr_against_hermite_kcrb_tgv64_matches_app_g(lbm):
    """The same case with KC-RR (App. G's Hermite-consistent reference):
    printed 0.061 % (E_k) and 0.314 % (Z) against Hermite KC-RB.  The
    difference is small (E_k: at most 1.6e-5 of u0^2), so each trajectory's
    own bound does not fix it; the GPU's difference r - h is therefore held
    sample by sample to the oracle's stored difference, within 1e-6 of that
    difference's largest magnitude (both are FP64 runs that differ only in
    rounding order; measured on a GB300: 1.8e-9 for E_k, 7.9e-10 for Z).
    The oracle's maxima (0.0623 % and 0.310 %) lie within 2.2 % of the printed
    values, so the GPU's do too; 10 % is asserted, as for the oracle."""
    gold = _gold()
    with open(os.path.join(GOLDEN, "kcrb_sensitivity_tgv64_oracle.json")) as fp:
        stored = json.load(fp)
    traj = _runs(lbm, ("hermite", "kcrr"))
    for key, printed in (("ek", gold["kcrr_vs_hermite_ek_max_rel_diff_percent"]),
                         ("z", gold["kcrr_vs_hermite_z_max_rel_diff_percent"])):
        h, r = traj["hermite"][key], traj["kcrr"][key]
        d_o = np.array(stored["kcrr"][key]) - np.array(stored["hermite"][key])
        drift = float(np.abs((r - h) - d_o).max() / np.abs(d_o).max())
        print(key, "GPU r-h against the oracle's, largest deviation / max|d|:", drift)
        assert drift <= 1e-6, (key, drift)
        got = 100 * float(np.max(np.abs(r - h) / np.abs(h)))
        assert got == pytest.approx(printed, rel=0.10), (key, got)
