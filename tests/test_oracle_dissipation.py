"""Pins of the oracle's dissipation rates (oracle.dissipation_pre / dissipation):
<2 rho nu_eff S:S> and <2 rho nu S:S> of a pre-collision state, nu_eff =
theta (1/omega_s - 1/2) from the closure's clipped rate (Eq.
omega_sgs_operational).

  - Shear wave u_x = U sin(2 pi z / N), rho = 1, at equilibrium: the central
    difference of Eq. (fd) gives S_xz = (U/2) sin(2 pi/N) cos(2 pi z/N) exactly,
    so <2 nu S:S> = nu U^2 sin^2(2 pi/N) / 2; m_neq = 0 and tr S = 0, so every
    closure's SGS trace vanishes, the rate is clipped and nu_eff = nu.
  - The same shear plus a trace mode alpha w_i (|c_i|^2 - 3 theta) (zero mass
    and momentum, uniform, so rho, u and S are unchanged): tr m_neq = 6 alpha
    theta^2 (fourth-order quadrature of D3Q27 and D3Q19), hence for KC-MP,
    KC-RB (both reconstructions) and KC-RR k = 3 |alpha| theta^2 and nu_eff =
    C_nu Delta sqrt(k) once that exceeds nu; BGK keeps nu.
  - dissipation() of a stored state equals dissipation_pre() of the same state
    pull-streamed by the independent numpy streaming of closure_data.
  - Planted mistakes in a copy of the C oracle (nu_eff without the -1/2, the
    factor 2 of 2 nu S:S, S:S without the off-diagonal terms) fail these pins.
"""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

THETA = 1.0 / 3.0
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _shear(orc, q, n, U, alpha=0.0):
    x = np.arange(n, dtype=np.float64)
    z = x[:, None, None] * np.ones((n, n, n))
    u = np.zeros((3, n, n, n))
    u[0] = U * np.sin(2 * math.pi * z / n)
    f = orc.init_equilibrium(q, None, u)
    if alpha:
        c, w, _ = orc.lattice(q)
        c2 = (c ** 2).sum(axis=1)
        f = f + (alpha * w * (c2 - 3 * THETA))[:, None, None, None]
    return f


def _exact_mol(nu, U, n):
    return nu * U * U * math.sin(2 * math.pi / n) ** 2 / 2


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("closure", [0, 1, 2, 3, 4])
def test_equilibrium_shear_dissipation(orc, q, closure):
    if closure == 4 and q == 19:
        pytest.skip("KC-RR is D3Q27 only")
    n, U, nu = 16, 0.02, 3e-3
    d = orc.dissipation_pre(_shear(orc, q, n, U), closure=closure, nu=nu, c_nu=0.035)
    ref = _exact_mol(nu, U, n)
    assert abs(d[1] - ref) <= 1e-13 * ref
    assert abs(d[0] - ref) <= 1e-13 * ref


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("closure", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("alpha", [2e-3, -2e-3])
def test_active_clip_dissipation(orc, q, closure, alpha):
    if closure == 4 and q == 19:
        pytest.skip("KC-RR is D3Q27 only")
    n, U, nu, c_nu = 16, 0.02, 1e-5, 0.035
    d = orc.dissipation_pre(_shear(orc, q, n, U, alpha), closure=closure, nu=nu, c_nu=c_nu)
    nu_t = c_nu * 1.0 * math.sqrt(3 * abs(alpha) * THETA ** 2)
    assert nu_t > nu
    nu_eff = nu if closure == 0 else nu_t
    assert abs(d[1] - _exact_mol(nu, U, n)) <= 1e-12 * _exact_mol(nu, U, n)
    assert abs(d[0] - _exact_mol(nu_eff, U, n)) <= 1e-12 * _exact_mol(nu_eff, U, n), (d, nu_eff)


def test_stored_state_is_streamed_first(orc):
    from oracle import closure_data

    rng = np.random.default_rng(3)
    from paper_2605_19796_gb300 import inputs

    rho, u = inputs.hit_fields(0, k0=2.0, urms=0.06, seed=4, shape=(12, 10, 8))
    f = orc.init_equilibrium(27, rho, u) * (1 + 1e-3 * rng.standard_normal((27, 8, 10, 12)))
    a = orc.dissipation(f, closure=1, nu=2e-5, c_nu=0.035)
    b = orc.dissipation_pre(closure_data.stream(f), closure=1, nu=2e-5, c_nu=0.035)
    assert np.abs(a - b).max() <= 1e-15 * np.abs(b).max()
    assert a[0] > a[1] > 0  # the closure is active: nu_eff > nu somewhere


MUTATIONS = [
    ("double nu_eff = ORC_THETA * (1.0 / omega_s - 0.5);", "double nu_eff = ORC_THETA * (1.0 / omega_s);"),
    ("e_eff = e_eff + 2.0 * rho[cidx] * nu_eff * ss;", "e_eff = e_eff + rho[cidx] * nu_eff * ss;"),
    ("for (int b = 0; b < 3; ++b) ss = ss + S[a][b] * S[a][b];", "ss = ss + S[a][a] * S[a][a];"),
]


@pytest.mark.parametrize("old,new", MUTATIONS)
def test_planted_mistakes_fail_the_pins(orc, tmp_path, old, new):
    src = open(os.path.join(ROOT, "oracle", "lbm_oracle.c")).read()
    assert old in src, old
    cpath, lpath = tmp_path / "mutant.c", tmp_path / "libmutant.so"
    cpath.write_text(src.replace(old, new))
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", str(cpath), "-o", str(lpath),
                    "-lm"], check=True)
    lib = ctypes.CDLL(str(lpath))
    dp, ip, c_int, c_double = (ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                               ctypes.c_double)
    lib.orc_dissipation_pre.argtypes = [c_int, c_int, c_int, c_int, c_int, ip, c_double, c_double, c_double, dp, dp, dp]

    def mutant_pre(f, closure, nu, c_nu):
        q, nz, ny, nx = f.shape
        ff = np.ascontiguousarray(f)
        bc = np.zeros(3, dtype=np.int32)
        F = np.zeros(3)
        out = np.zeros(2)
        rc = lib.orc_dissipation_pre(q, nx, ny, nz, closure, bc.ctypes.data_as(ip), nu, c_nu, 1.0,
                                     F.ctypes.data_as(dp), ff.ctypes.data_as(dp), out.ctypes.data_as(dp))
        assert rc == 0
        return out

    n, U = 16, 0.02
    failed = False
    for alpha, nu in ((0.0, 3e-3), (2e-3, 1e-5)):
        d = mutant_pre(_shear(orc, 27, n, U, alpha), 1, nu, 0.035)
        nu_eff = nu if alpha == 0 else 0.035 * math.sqrt(3 * alpha * THETA ** 2)
        if abs(d[0] - _exact_mol(nu_eff, U, n)) > 1e-12 * _exact_mol(nu_eff, U, n) or \
                abs(d[1] - _exact_mol(nu, U, n)) > 1e-12 * _exact_mol(nu, U, n):
            failed = True
    assert failed, "the planted mistake passed the pins"
