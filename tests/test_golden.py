"""Values the paper prints, kept as cited text fixtures under tests/golden/
(no GPU): the lattice constants of App. F, the closure constants of Sec. 7,
the App. G comparison of the two KC-RB reconstructions on the 64^3
Taylor-Green vortex, which the FP64 oracle reproduces, and the Sec. 7.1
statement that at N = 128 the closures follow the resolved-BGK energy curve
(the oracle trajectories are stored by the make_*.py scripts beside the
fixtures, and their first steps are re-run here to tie the stored files to
the current oracle)."""
import importlib.util
import json
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name):
    """key -> value of a fixture file (comments start with #)."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as fp:
        for line in fp:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split()
                out[k] = v
    return out


def _maker():
    spec = importlib.util.spec_from_file_location("make_kcrb_sensitivity",
                                                  os.path.join(GOLDEN, "make_kcrb_sensitivity.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_lattice_constants_as_printed(orc):
    g = read_golden("lattice_constants.txt")
    theta = Fraction(g["theta_R"])
    w1d = {0: Fraction(g["w1d_0"]), 1: Fraction(g["w1d_pm1"])}
    assert orc.THETA == float(theta)
    for q in (27,):
        c, w, _ = orc.lattice(q)
        for i in range(q):
            exact = w1d[abs(c[i, 0])] * w1d[abs(c[i, 1])] * w1d[abs(c[i, 2])]
            assert abs(w[i] - float(exact)) <= 1e-16 * float(exact) + 1e-18
        assert sum(Fraction(w1d[abs(a)]) * w1d[abs(b)] * w1d[abs(d)] for a, b, d in c) == 1


def test_closure_constants_as_printed():
    from paper_2605_19796_gb300 import build

    build.build()
    from paper_2605_19796_gb300 import lbm

    g = read_golden("closure_cnu.txt")
    for name, v in g.items():
        assert lbm.DEFAULT_CNU[lbm.CLOSURES[name]] == float(v), name
    cfg = lbm.lbm_config()
    lbm.LIB.lbm_config_default(cfg)
    assert cfg.closure == lbm.CLOSURES["kcmp"] and cfg.c_nu == float(g["kcmp"])


def _sensitivity(traj):
    """max over the window of |raw - hermite| / |hermite| (E_k, Z) and whether
    each difference takes both signs."""
    res = {}
    for key in ("ek", "z"):
        h, r = np.array(traj["hermite"][key]), np.array(traj["raw"][key])
        d = r - h
        res[key] = (float(np.max(np.abs(d) / np.abs(h))), bool((d > 0).any() and (d < 0).any()))
    return res


def test_kcrb_sensitivity_of_the_oracle_matches_app_g():
    """The oracle's maximum relative differences between KC-RB raw and
    Hermite on the App. G Taylor-Green case (stored trajectories) against the
    printed 3.06 % (E_k) and 12.82 % (Z), and both differences change sign.
    Bounds: 2 % of the printed E_k value and 3 % of the Z value, whose maximum
    sits at the end of the window (so it depends on where the paper stopped
    and how finely it sampled)."""
    g = read_golden("kcrb_sensitivity_tgv64.txt")
    with open(os.path.join(GOLDEN, "kcrb_sensitivity_tgv64_oracle.json")) as fp:
        traj = json.load(fp)
    res = _sensitivity(traj)
    ek, z = 100 * res["ek"][0], 100 * res["z"][0]
    assert ek == pytest.approx(float(g["ek_max_rel_diff_percent"]), rel=0.02), ek
    assert z == pytest.approx(float(g["z_max_rel_diff_percent"]), rel=0.03), z
    assert res["ek"][1] and res["z"][1] and g["both_change_sign"] == "1"
    assert traj["hermite"]["t"][-1] > 19.9


def test_kcrr_against_hermite_kcrb_matches_app_g():
    """App. G's contextual reference: KC-RR (C_nu = 0.02) against Hermite
    KC-RB on the same case, printed maximum relative differences 0.061 %
    (E_k) and 0.314 % (Z); the oracle's stored trajectories within 10 % of
    each (a bound chosen before the KC-RR run; the oracle gives 0.0623 % and
    0.310 %)."""
    g = read_golden("kcrb_sensitivity_tgv64.txt")
    with open(os.path.join(GOLDEN, "kcrb_sensitivity_tgv64_oracle.json")) as fp:
        traj = json.load(fp)
    for key, name in (("ek", "kcrr_vs_hermite_ek_max_rel_diff_percent"),
                      ("z", "kcrr_vs_hermite_z_max_rel_diff_percent")):
        h, r = np.array(traj["hermite"][key]), np.array(traj["kcrr"][key])
        got = 100 * float(np.max(np.abs(r - h) / np.abs(h)))
        assert got == pytest.approx(float(g[name]), rel=0.10), (key, got)


def test_stored_sensitivity_trajectories_are_the_oracles():
    """The first steps of the three App. G runs (60 for the KC-RB pair, 20 for
    the slower KC-RR), re-run with the current oracle, equal the stored
    trajectories (FP64, same arithmetic)."""
    mk = _maker()
    with open(os.path.join(GOLDEN, "kcrb_sensitivity_tgv64_oracle.json")) as fp:
        traj = json.load(fp)
    for name, closure, steps in (("hermite", 2, 60), ("raw", 3, 60), ("kcrr", 4, 20)):
        now = mk.trajectory(closure, steps_max=steps)
        k = len(now["ek"])
        for key in ("t", "ek", "z"):
            a, b = np.array(now[key]), np.array(traj[name][key][:k])
            assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max(), (name, key)


def _clip_window_and_diff(t64, b64, k64, t128, b128, k128):
    """The window of tgv128_clip.txt (t up to the first sample where the N = 64
    BGK kinetic energy exceeds its running minimum by 1 %) and D(64), D(128)
    over it."""
    b64, k64 = np.asarray(b64), np.asarray(k64[: len(b64)])
    t64 = np.asarray(t64[: len(b64)])
    run_min = np.minimum.accumulate(b64)
    grow = np.nonzero((b64 - run_min) / run_min > 0.01)[0]
    t_end = t64[grow[0]] if len(grow) else t64[-1]
    m64 = t64 <= t_end
    d64 = float(np.max(np.abs(k64[m64] - b64[m64]) / b64[m64]))
    t128, b128, k128 = np.asarray(t128), np.asarray(b128), np.asarray(k128)
    m128 = t128 <= t_end
    d128 = float(np.max(np.abs(k128[m128] - b128[m128]) / b128[m128]))
    return t_end, d64, d128


def test_tgv128_closure_follows_bgk_as_sec_7_1_states():
    """Sec. 7.1: at N = 128 the rate limiter clips the SGS relaxation almost
    everywhere, so KC-MP's kinetic energy follows the resolved-BGK curve far
    more closely than at N = 64 (stored oracle trajectories at both
    resolutions; the ratio criterion of tgv128_clip.txt)."""
    g = read_golden("tgv128_clip.txt")
    with open(os.path.join(GOLDEN, "tgv128_clip_oracle.json")) as fp:
        t128 = json.load(fp)
    with open(os.path.join(GOLDEN, "tgv64_clip_oracle.json")) as fp:
        t64 = json.load(fp)
    assert t128["bgk"]["t"][-1] > 19.9
    t_end, d64, d128 = _clip_window_and_diff(t64["bgk"]["t"], t64["bgk"]["ek"], t64["kcmp"]["ek"],
                                             t128["bgk"]["t"], t128["bgk"]["ek"], t128["kcmp"]["ek"])
    assert 9.0 < t_end < 11.3, t_end
    assert d64 / d128 >= float(g["n64_over_n128_ratio_at_least"]), (d64, d128)


def test_stored_tgv64_trajectories_are_the_oracles():
    """The first 20 steps of both N = 64 runs, re-run with the current oracle,
    equal the stored trajectories; the stored BGK run ends where it turns
    non-finite (before t u0/L = 12) while KC-MP runs to the end."""
    spec = importlib.util.spec_from_file_location("make_tgv64_clip", os.path.join(GOLDEN, "make_tgv64_clip.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    with open(os.path.join(GOLDEN, "tgv64_clip_oracle.json")) as fp:
        traj = json.load(fp)
    for name, closure, c_nu in mk.RUNS:
        now = mk.trajectory(closure, c_nu, steps_max=20)
        k = len(now["ek"])
        for key in ("t", "ek"):
            a, b = np.array(now[key]), np.array(traj[name][key][:k])
            assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max(), (name, key)
    assert traj["bgk"]["t"][-1] < 11.5 < traj["kcmp"]["t"][-1]


def test_stored_tgv128_trajectories_are_the_oracles():
    """The first 20 steps of both N = 128 runs, re-run with the current
    oracle, equal the stored trajectories."""
    spec = importlib.util.spec_from_file_location("make_tgv128_clip", os.path.join(GOLDEN, "make_tgv128_clip.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    with open(os.path.join(GOLDEN, "tgv128_clip_oracle.json")) as fp:
        traj = json.load(fp)
    for name, closure, c_nu in mk.RUNS:
        now = mk.trajectory(closure, c_nu, steps_max=20)
        k = len(now["ek"])
        for key in ("t", "ek", "z"):
            a, b = np.array(now[key]), np.array(traj[name][key][:k])
            assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max(), (name, key)
