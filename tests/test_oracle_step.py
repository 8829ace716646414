"""Pins of the oracle's full time step (no GPU).

  - macroscopic fields (App. F.1 step 1) against brute-force loops on a 4^3 lattice;
  - the streaming direction of Eq. (streaming) in pull form;
  - the finite-difference strain, Eqs. (fd), (fd_boundary_lower/upper),
    (strain_rate_discrete): exact on quadratic fields, second order on sines;
  - global conservation of mass and momentum over many steps;
  - the resolved-BGK limit over a whole run (C_nu = 0 reproduces BGK);
  - exact Navier-Stokes decays at low Reynolds number (shear wave
    exp(-nu k^2 t) with second-order convergence; 2D Taylor-Green energy
    exp(-4 nu k^2 t)), where the clip of Eq. (omega_sgs_operational) makes
    the closures reduce to BGK;
  - the x<->y mirror symmetry of the 3D Taylor-Green vortex;
  - the moments of Guo's forcing source (mass kept, momentum + F, second
    moment + (1 - omega/2)(u F + F u));
  - laminar Poiseuille flow with bounce-back walls and a body force;
  - the Sec. 7.1 diagnostics on the Taylor-Green initial field, and on a
    general band-limited field with varying density (enstrophy against the
    Fourier-space curl);
  - the single-cell step against the full-lattice step.
"""
import itertools
import math

import numpy as np
import pytest

from paper_2605_19796_gb300 import inputs

THETA = 1.0 / 3.0
EPS = np.finfo(float).eps


def _velocities(q):
    """Canonical order written out from its rule: cz outer, cy, cx fastest."""
    out = []
    for cz, cy, cx in itertools.product((-1, 0, 1), repeat=3):
        if q == 19 and abs(cx) + abs(cy) + abs(cz) == 3:
            continue
        out.append((cx, cy, cz))
    return out


@pytest.mark.parametrize("q", [19, 27])
def test_fields_brute_force(orc, q):
    f = inputs.random_populations(q, (4, 4, 4), seed=1, amp=0.3)
    rho, u = orc.fields(f)
    vel = _velocities(q)
    for z in range(4):
        for y in range(4):
            for x in range(4):
                r = 0.0
                m = [0.0, 0.0, 0.0]
                for i, c in enumerate(vel):
                    r += f[i, z, y, x]
                    for a in range(3):
                        m[a] += f[i, z, y, x] * c[a]
                assert rho[z, y, x] == pytest.approx(r, rel=1e-15)
                for a in range(3):
                    assert u[a, z, y, x] == pytest.approx(m[a] / r, rel=1e-13, abs=1e-17)


@pytest.mark.parametrize("q", [19, 27])
def test_streaming_direction(orc, q):
    """With nu -> infinity, omega_hat -> 0 and one step is pure streaming:
    f_i(x) <- f_i(x - c_i) (periodic)."""
    shape = (5, 4, 3)
    f = inputs.random_populations(q, shape, seed=2, amp=0.3)
    g = orc.run(f, 1, closure=0, nu=1e12)
    vel = _velocities(q)
    for i, (cx, cy, cz) in enumerate(vel):
        expect = np.roll(f[i], shift=(cz, cy, cx), axis=(0, 1, 2))
        assert np.abs(g[i] - expect).max() < 1e-11


def test_strain_exact_on_quadratics_with_walls(orc):
    """Central and one-sided second-order formulas are exact for quadratics."""
    nx, ny, nz = 6, 5, 7
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    rng = np.random.default_rng(0)
    coef = rng.standard_normal((3, 10))

    def poly(cf):
        return (cf[0] + cf[1] * x + cf[2] * y + cf[3] * z + cf[4] * x * x + cf[5] * y * y + cf[6] * z * z
                + cf[7] * x * y + cf[8] * y * z + cf[9] * x * z)

    def dpoly(cf, axis):
        if axis == 0:
            return cf[1] + 2 * cf[4] * x + cf[7] * y + cf[9] * z
        if axis == 1:
            return cf[2] + 2 * cf[5] * y + cf[7] * x + cf[8] * z
        return cf[3] + 2 * cf[6] * z + cf[8] * y + cf[9] * x

    u = np.stack([poly(coef[b]) for b in range(3)]).astype(float)
    S = orc.strain_field(u, bc=(1, 1, 1))
    for a in range(3):
        for b in range(3):
            ref = 0.5 * (dpoly(coef[a], b) + dpoly(coef[b], a))
            assert np.abs(S[a, b] - ref).max() < 1e-12


def test_strain_second_order_periodic(orc):
    errs = []
    for n in (16, 32, 64):
        x = np.arange(n)
        u = np.zeros((3, 1, 1, n))
        u[1, 0, 0, :] = np.sin(2 * math.pi * x / n)
        S = orc.strain_field(u)
        ref = 0.5 * (2 * math.pi / n) * np.cos(2 * math.pi * x / n)
        errs.append(np.abs(S[0, 1, 0, 0] - ref).max() / np.abs(ref).max())
        assert np.abs(S[0, 1] - S[1, 0]).max() == 0.0
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.02)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.02)


def _hit_pops(orc, q, n, seed=0, urms=0.04):
    rho, u = inputs.hit_fields(n, k0=2.0, urms=urms, seed=seed)
    return orc.init_equilibrium(q, rho, u)


@pytest.mark.parametrize("q,closure", [(19, 1), (27, 1), (19, 2), (27, 0), (27, 4)])
def test_global_conservation(orc, q, closure):
    f = _hit_pops(orc, q, 10, seed=3, urms=0.08)
    c = np.array(_velocities(q), dtype=float)
    m0 = f.sum()
    p0 = np.einsum("iabc,ik->k", f, c)
    g = orc.run(f, 40, closure=closure, nu=2e-5, c_nu=0.035)
    assert abs(g.sum() - m0) / m0 < 1e-13
    assert np.abs(np.einsum("iabc,ik->k", g, c) - p0).max() < 1e-13 * m0 * 0.08


@pytest.mark.parametrize("closure", [1, 2, 3])
def test_run_resolved_bgk_limit(orc, closure):
    f = _hit_pops(orc, 27, 8, seed=4, urms=0.08)
    a = orc.run(f, 20, closure=0, nu=2e-5)
    b = orc.run(f, 20, closure=closure, nu=2e-5, c_nu=0.0)
    assert np.abs(a - b).max() < 1e-14


def test_closure_active_under_resolution(orc):
    """At low resolution and high Reynolds number the turbulent rate is active and
    KC-MP departs from BGK; it stays conservative."""
    f = _hit_pops(orc, 27, 8, seed=4, urms=0.08)
    a = orc.run(f, 20, closure=0, nu=2e-5)
    b = orc.run(f, 20, closure=1, nu=2e-5, c_nu=0.035)
    assert np.abs(a - b).max() > 1e-6


def _shear_amplitudes(orc, q, n, nu, steps, closure=1):
    rho, u = inputs.shear_wave_fields(n, amp=1e-4, nxy=1)
    g = orc.init_equilibrium(q, rho, u)
    z = np.arange(n)
    s = np.sin(2 * math.pi * z / n)
    out = []
    for st in steps:
        g = orc.run(g, st, closure=closure, nu=nu, c_nu=0.035)
        _, ug = orc.fields(g)
        out.append(float(ug[0, :, 0, 0] @ s / (s @ s)) / 1e-4)
    return out


@pytest.mark.parametrize("q", [19, 27])
def test_shear_wave_decay(orc, q):
    """u_x = A sin(k z) decays as exp(-nu k^2 t) (exact Navier-Stokes).  The rate
    is measured between t1 = T/4 and T (after the transient of the
    equilibrium-only initial state); its lattice error converges at second
    order in k (diffusive scaling, nu fixed)."""
    nu = 0.05
    errs = []
    for n in (16, 32, 64):
        k = 2 * math.pi / n
        T = int(round(0.5 / (nu * k * k)))
        a1, a2 = _shear_amplitudes(orc, q, n, nu, [T // 4, T - T // 4])
        rate = -math.log(a2 / a1) / (T - T // 4)
        errs.append(abs(rate / (nu * k * k) - 1.0))
    assert errs[2] < 1e-3
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.05)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.05)


def test_shear_wave_tau_one_is_fourth_order(orc):
    """At nu = 1/6 (tau_hat = 1) the BGK shear-wave error is fourth order (a
    known property of the lattice BGK scheme)."""
    errs = []
    for n in (16, 32):
        nu = 1.0 / 6.0
        k = 2 * math.pi / n
        T = int(round(0.5 / (nu * k * k)))
        a1, a2 = _shear_amplitudes(orc, 27, n, nu, [T // 4, T - T // 4])
        errs.append(abs(-math.log(a2 / a1) / (T - T // 4) / (nu * k * k) - 1.0))
    assert errs[0] < 1e-4 and errs[0] / errs[1] > 12.0


@pytest.mark.parametrize("q,closure", [(19, 1), (27, 1), (27, 2), (27, 4)])
def test_tgv2d_energy_decay(orc, q, closure):
    """2D Taylor-Green: E(t) = E0 exp(-4 nu k^2 t), k = 2 pi / n."""
    n, nu, steps = 32, 0.02, 400
    c_nu = 0.035 if closure == 1 else 0.02
    rho, u = inputs.tgv2d_fields(n, u0=0.01, nz=1)
    f = orc.init_equilibrium(q, rho, u)
    g = orc.run(f, 100, closure=closure, nu=nu, c_nu=c_nu)  # past the initial transient
    e1 = orc.diagnostics(g)[4]
    g = orc.run(g, steps, closure=closure, nu=nu, c_nu=c_nu)
    e2 = orc.diagnostics(g)[4]
    k = 2 * math.pi / n
    assert e2 / e1 == pytest.approx(math.exp(-4 * nu * k * k * steps), rel=5e-4)


@pytest.mark.parametrize("q", [19, 27])
def test_tgv3d_symmetries(orc, q):
    """Symmetries of the TGV that Navier-Stokes and the lattice preserve:
    the mirror x -> -x (u_x odd, u_y, u_z, rho even) and the swap
    (x, y, z) -> (y, x, z + L/2) with (u_x, u_y) exchanged."""
    n = 12
    rho, u = inputs.tgv_fields(n, u0=0.05)
    f = orc.init_equilibrium(q, rho, u)
    g = orc.run(f, 30, closure=1, nu=3e-4, c_nu=0.035)
    r, ug = orc.fields(g)
    assert np.abs(ug).max() > 0.04
    mx = lambda a: a[..., (-np.arange(n)) % n]
    assert np.abs(mx(r) - r).max() < 1e-13
    assert np.abs(mx(ug[0]) + ug[0]).max() < 1e-13
    assert np.abs(mx(ug[1]) - ug[1]).max() < 1e-13
    sw = lambda a: np.roll(np.swapaxes(a, -1, -2), -n // 2, axis=0)
    assert np.abs(sw(r) - r).max() < 1e-13
    assert np.abs(sw(ug[0]) - ug[1]).max() < 1e-13
    assert np.abs(sw(ug[1]) - ug[0]).max() < 1e-13
    assert np.abs(sw(ug[2]) - ug[2]).max() < 1e-13


@pytest.mark.parametrize("q", [19, 27])
def test_guo_source_moments(orc, q):
    """With a body force the collision adds Guo's source (the reading taken
    where the paper neglects forces): after a BGK collision the mass is
    unchanged, the momentum has gained F, and the second moment is the
    unforced relaxation of Pi towards rho (u u + theta I), u = (sum f c +
    F/2)/rho, plus (1 - omega/2)(u F + F u), the second moment of the textbook
    source, which follows from the fourth-order isotropy both lattices have."""
    rng = np.random.default_rng(31)
    c = np.array(_velocities(q), dtype=float)
    _, w, _ = orc.lattice(q)
    for k in range(4):
        f = w * (1.0 + 0.05 * rng.standard_normal(q))
        F = 1e-3 * rng.standard_normal(3)
        nu = 0.02 + 0.05 * k
        omega = 1.0 / (nu / THETA + 0.5)
        fp, _ = orc.collide_cell(q, 0, f, np.zeros((3, 3)), nu, 0.0, F=F)
        rho = f.sum()
        u = (f @ c + 0.5 * F) / rho
        pi = np.einsum("i,ia,ib->ab", f, c, c)
        want = pi - omega * (pi - rho * (np.outer(u, u) + THETA * np.eye(3))) + (1 - 0.5 * omega) * (
            np.outer(u, F) + np.outer(F, u))
        assert np.abs(np.einsum("i,ia,ib->ab", fp, c, c) - want).max() <= 1e-15
        assert abs(fp.sum() - rho) <= 4 * EPS
        assert np.abs(fp @ c - (f @ c + F)).max() <= 1e-16


@pytest.mark.parametrize("q", [19, 27])
def test_poiseuille_bounce_back(orc, q):
    """Body-forced flow between halfway bounce-back walls in y (walls at y = -1/2
    and y = ny - 1/2) relaxes to u_x(y) = F/(2 rho nu) (y + 1/2)(ny - 1/2 - y);
    the discrete profile error shrinks at second order."""
    errs = []
    for ny in (8, 16):
        nu = 0.1
        F = 1e-6 * (8.0 / ny) ** 2
        u = np.zeros((3, 1, ny, 1))
        f = orc.init_equilibrium(q, None, u)
        H = float(ny)
        steps = int(3.0 * H * H / nu)
        g = orc.run(f, steps, closure=1, nu=nu, c_nu=0.035, bc=(0, 1, 0), F=(F, 0.0, 0.0))
        _, ug = orc.fields(g, F=(F, 0.0, 0.0))
        y = np.arange(ny) + 0.5
        ref = F / (2 * nu) * y * (H - y)
        errs.append(np.abs(ug[0, 0, :, 0] - ref).max() / ref.max())
    assert errs[1] < 0.02
    assert errs[0] / errs[1] > 3.0


def test_enstrophy_of_a_general_field(orc):
    """Diagnostics (Sec. 7.1) of a band-limited periodic field whose three
    velocity components vary along all three axes, with a varying density:
    mass and momentum against the populations' sums, E_k = <rho |u|^2 / 2>,
    and the enstrophy against the curl taken exactly in Fourier space.  The sixth-order central differences differ from the exact
    derivative by about (k dx)^6 / 140 of it at the largest wavenumber here
    (k dx = 0.52: 1.5e-4), so 2e-3 of the enstrophy bounds the difference."""
    n = 24
    rng = np.random.default_rng(77)
    x = 2 * math.pi * np.arange(n) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    u = np.zeros((3, n, n, n))
    modes = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (0, 1, 1), (1, 0, 1), (2, 1, 0), (0, 2, 1), (1, -1, 2)]
    for a in range(3):
        for kx, ky, kz in modes:
            u[a] += 0.01 * rng.standard_normal() * np.sin(kx * X + ky * Y + kz * Z + rng.uniform(0, 2 * math.pi))
    rho = 1.0 + 2.0 * u.sum(axis=0)  # correlated with u, so rho u and rho |u|^2 differ from u and |u|^2
    f = orc.init_equilibrium(27, rho, u)
    d = orc.diagnostics(f)
    # mass and momentum: the populations' own sums
    c, _, _ = orc.lattice(27)
    assert d[0] == pytest.approx(f.sum(), rel=1e-14)
    assert np.abs(d[1:4] - np.einsum("iabc,ik->k", f, c.astype(float))).max() <= 1e-14 * np.abs(u).sum()
    k = 2 * math.pi * np.fft.fftfreq(n)
    uh = np.fft.fftn(u, axes=(1, 2, 3))
    kk = {0: k[None, None, :], 1: k[None, :, None], 2: k[:, None, None]}  # d/dx, d/dy, d/dz on [z, y, x]

    def d_(comp, axis):
        return np.real(np.fft.ifftn(1j * kk[axis] * uh[comp]))

    wx = d_(2, 1) - d_(1, 2)
    wy = d_(0, 2) - d_(2, 0)
    wz = d_(1, 0) - d_(0, 1)
    zz = np.mean(0.5 * (wx ** 2 + wy ** 2 + wz ** 2))
    assert d[5] == pytest.approx(zz, rel=2e-3)
    assert d[4] == pytest.approx(np.mean(0.5 * rho * (u ** 2).sum(axis=0)), rel=1e-12)


def test_diagnostics_tgv_initial(orc):
    """E_k and enstrophy of the TGV initial field against their exact discrete /
    continuum values (sixth-order curl error ~ (2 pi / n)^6)."""
    n, u0 = 32, 0.05
    rho, u = inputs.tgv_fields(n, u0=u0)
    f = orc.init_equilibrium(27, rho, u)
    d = orc.diagnostics(f)
    assert d[0] == pytest.approx(rho.sum(), rel=1e-14)
    ek = np.mean(0.5 * rho * (u ** 2).sum(axis=0))
    assert d[4] == pytest.approx(ek, rel=1e-12)
    # continuum vorticity of the TGV: enstrophy mean = (3/8) u0^2 k^2 ... computed here from the analytic curl
    k = 2 * math.pi / n
    X = k * np.arange(n)
    Z, Y, Xg = np.meshgrid(X, X, X, indexing="ij")
    wx = -u0 * k * np.cos(Xg) * np.sin(Y) * np.sin(Z)
    wy = -u0 * k * np.sin(Xg) * np.cos(Y) * np.sin(Z)
    wz = 2 * u0 * k * np.sin(Xg) * np.sin(Y) * np.cos(Z)
    zz = np.mean(0.5 * (wx ** 2 + wy ** 2 + wz ** 2))
    assert zz == pytest.approx(0.375 * u0 ** 2 * k ** 2, rel=1e-12)
    assert d[5] == pytest.approx(zz, rel=5 * k ** 6)
    assert d[6] == 0.0


@pytest.mark.parametrize("closure", [0, 1, 2, 3, 4])
def test_step_cell_matches_full_step(orc, closure):
    q = 27
    f = _hit_pops(orc, q, 7, seed=5, urms=0.08)
    g = orc.run(f, 1, closure=closure, nu=2e-5, c_nu=0.035)
    rng = np.random.default_rng(0)
    for _ in range(6):
        x, y, z = rng.integers(0, 7, size=3)
        idx = np.ix_(range(q), (z + np.arange(-2, 3)) % 7, (y + np.arange(-2, 3)) % 7, (x + np.arange(-2, 3)) % 7)
        blk = f[idx]
        out = orc.step_cell(blk, closure=closure, nu=2e-5, c_nu=0.035)
        assert np.abs(out - g[:, z, y, x]).max() < 1e-15
