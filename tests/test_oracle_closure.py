"""Pins of the oracle's collision and closure (no GPU).

Each test states the passage of the paper (or the mathematical fact) it checks:
  - f_sgs has zero zeroth and first moments, Eqs. (f_sgs_zero_moment),
    (f_sgs_first_moment); KC-MP's second moment reproduces m_sgs (projection
    of Eq. f_sgs_KCMP with the quadrature identity of the lattice);
  - the KC-RB CE reconstruction has zero mass and momentum, and its second
    moment is the CE stress m^CE = -2 rho theta tau_hat S (App. F.3);
  - raw vs Hermite KC-RB: f1_raw = f1 - w rho tau_hat div u (App. F.2);
  - raw KC-RB mass defect sum(f_post - f) = (omega - omega_s) rho tau_hat div u;
  - the collision conserves mass and momentum (App. F.1, "filtered-density and
    filtered-momentum conserving") for BGK, KC-MP, Hermite KC-RB and KC-RR;
  - the resolved-BGK limit omega_s = omega reproduces BGK (Sec. 5.1,
    "The resolved BGK limit"; for KC-RR, Sec. 7.1: the full D3Q27
    representation recombines);
  - the trapezoidal reconstruction of App. F.5 (Eq. correct_Qi): the explicit
    two-rate update solves the implicit relation with tau in the unshifted CE part;
  - the rate formula Eq. (omega_sgs_operational);
  - KC-RR on a state built from its Hermite coefficients, against the closed
    form of the RR recursion Eq. (kcrr_rr) and the two-rate relaxation of
    App. F.4.
"""
import numpy as np
import pytest

THETA = 1.0 / 3.0
EPS = np.finfo(float).eps
# round-off bound for a sum of q = 27 terms of size <= 1 computed in FP64
TOL = 32 * EPS
CLOSURES = {"bgk": 0, "kcmp": 1, "kcrb_h": 2, "kcrb_raw": 3, "kcrr": 4}


def _state(orc, q, seed, amp=0.02, neq=0.01):
    """Random near-equilibrium populations (neq content large enough that the
    turbulent rate is active) and a random symmetric strain."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.05 * rng.standard_normal()
    u = amp * rng.standard_normal(3)
    f = orc.equilibrium(q, rho, u)
    _, w, _ = orc.lattice(q)
    f = f + neq * w * rng.standard_normal(q)
    # keep rho and rho u of f equal to those used above: remove the noise's
    # zeroth and first moments
    c = orc.lattice(q)[0].astype(float)
    d0 = f.sum() - rho
    d1 = f @ c - rho * u
    f = f - w * d0 - w * (c @ d1) / THETA
    A = 0.01 * rng.standard_normal((3, 3))
    S = 0.5 * (A + A.T)
    return f, S, rho, u


def _cq(orc, q):
    return orc.lattice(q)[0].astype(float)


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("seed", range(4))
def test_kcmp_carrier_moments(orc, q, seed):
    f, S, rho, u = _state(orc, q, seed)
    nu = 1e-3
    f0, f1, fsgs, om_s = orc.closure_parts(q, CLOSURES["kcmp"], f, S, nu, 0.035)
    c = _cq(orc, q)
    assert abs(fsgs.sum()) < TOL * np.abs(fsgs).max()
    assert np.abs(fsgs @ c).max() < TOL * np.abs(fsgs).max()
    tau_hat = 1.0 / orc.omega_hat(nu)
    mneq = np.einsum("i,ia,ib->ab", f - f0, c, c)
    msgs = mneq - (-2.0 * rho * THETA * tau_hat * S)
    assert np.abs(np.einsum("i,ia,ib->ab", fsgs, c, c) - msgs).max() < TOL * np.abs(f - f0).max()
    # f1 carries exactly the CE stress
    assert np.abs(np.einsum("i,ia,ib->ab", f1, c, c) - (-2.0 * rho * THETA * tau_hat * S)).max() < TOL * np.abs(f - f0).max()


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("seed", range(4))
def test_kcrb_hermite_ce_part(orc, q, seed):
    f, S, rho, u = _state(orc, q, seed)
    nu = 1e-3
    tau_hat = 1.0 / orc.omega_hat(nu)
    f0, f1, fsgs, _ = orc.closure_parts(q, CLOSURES["kcrb_h"], f, S, nu, 0.02)
    c = _cq(orc, q)
    sc = np.abs(f1).max()
    assert abs(f1.sum()) < TOL * sc and np.abs(f1 @ c).max() < TOL * sc
    assert np.abs(np.einsum("i,ia,ib->ab", f1, c, c) - (-2.0 * rho * THETA * tau_hat * S)).max() < TOL * sc
    # carrier definition, Eq. (kcrb_operational_fsgs)
    assert np.abs(fsgs - (f - f0 - f1)).max() < 4 * EPS * np.abs(f).max()


@pytest.mark.parametrize("q", [19, 27])
def test_kcrb_raw_vs_hermite(orc, q):
    f, S, rho, u = _state(orc, q, 11)
    nu = 1e-5
    tau_hat = 1.0 / orc.omega_hat(nu)
    _, w, _ = orc.lattice(q)
    _, f1h, _, _ = orc.closure_parts(q, CLOSURES["kcrb_h"], f, S, nu, 0.02)
    _, f1r, _, om_s = orc.closure_parts(q, CLOSURES["kcrb_raw"], f, S, nu, 0.02)
    assert np.abs(f1r - (f1h - w * rho * tau_hat * np.trace(S))).max() < TOL * np.abs(f1h).max()
    # mass defect of the raw form
    fpost, om_s2 = orc.collide_cell(q, CLOSURES["kcrb_raw"], f, S, nu, 0.02)
    assert om_s < orc.omega_hat(nu), "test state must activate the turbulent rate"
    om = orc.omega_hat(nu)
    assert om_s2 == om_s and om_s < om
    assert (fpost.sum() - f.sum()) == pytest.approx((om - om_s) * rho * tau_hat * np.trace(S), rel=1e-9)


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("name", ["bgk", "kcmp", "kcrb_h", "kcrr"])
@pytest.mark.parametrize("seed", range(3))
def test_collision_conserves(orc, q, name, seed):
    if name == "kcrr" and q == 19:
        pytest.skip("KC-RR is defined on D3Q27 only")
    f, S, rho, u = _state(orc, q, seed)
    nu = 1e-5
    fpost, om_s = orc.collide_cell(q, CLOSURES[name], f, S, nu, 0.035)
    if name != "bgk":
        assert om_s < orc.omega_hat(nu), "test state must activate the turbulent rate"
    c = _cq(orc, q)
    assert abs(fpost.sum() - f.sum()) < TOL
    assert np.abs(fpost @ c - f @ c).max() < TOL


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("name", ["kcmp", "kcrb_h", "kcrb_raw", "kcrr"])
def test_resolved_bgk_limit(orc, q, name):
    """C_nu = 0 gives omega_s = omega exactly, and the update equals BGK to round-off."""
    if name == "kcrr" and q == 19:
        pytest.skip("KC-RR is defined on D3Q27 only")
    f, S, rho, u = _state(orc, q, 3)
    nu = 1e-3
    bgk, _ = orc.collide_cell(q, 0, f, S, nu, 0.0)
    got, om_s = orc.collide_cell(q, CLOSURES[name], f, S, nu, 0.0)
    assert om_s == orc.omega_hat(nu)
    assert np.abs(got - bgk).max() < TOL * np.abs(f).max()


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("name", ["bgk", "kcmp", "kcrb_h", "kcrb_raw", "kcrr"])
def test_uniform_flow_is_fixed_point(orc, q, name):
    if name == "kcrr" and q == 19:
        pytest.skip("KC-RR is defined on D3Q27 only")
    f = orc.equilibrium(q, 1.02, [0.03, -0.01, 0.02])
    got, om_s = orc.collide_cell(q, CLOSURES[name], f, np.zeros((3, 3)), 1e-4, 0.035)
    assert np.abs(got - f).max() < TOL * np.abs(f).max()


def test_kcmp_ignores_moments_above_second(orc):
    """KC-MP's carrier depends on f only through its second moment (Sec. 6.3):
    adding a third-order Hermite mode to f leaves f_sgs unchanged."""
    q = 27
    f, S, rho, u = _state(orc, q, 5)
    c = _cq(orc, q)
    _, w, _ = orc.lattice(q)
    g = f + 1e-3 * w * (c[:, 0] ** 2 - THETA) * c[:, 1]  # H_xxy, zero moments up to order 2
    _, _, fsgs_a, _ = orc.closure_parts(q, 1, f, S, 1e-3, 0.035)
    _, _, fsgs_b, _ = orc.closure_parts(q, 1, g, S, 1e-3, 0.035)
    # f - f0 is formed from O(|f|) values, so round-off scales with |f|
    assert np.abs(fsgs_a - fsgs_b).max() < TOL * np.abs(f).max()


def test_kcrr_relaxes_high_order_modes(orc):
    """KC-RR at omega_s = omega is BGK of the complete D3Q27 Hermite content
    (Sec. 7.1); with omega_s < omega the third-order SGS departure from the RR
    manifold is relaxed more slowly than the RR part, so the KC-RR and BGK
    updates differ in the H_xxy moment but agree in mass and momentum."""
    q = 27
    f, S, rho, u = _state(orc, q, 7)
    c = _cq(orc, q)
    bgk, _ = orc.collide_cell(q, 0, f, S, 1e-5, 0.035)
    rr, om_s = orc.collide_cell(q, 4, f, S, 1e-5, 0.035)
    assert om_s < orc.omega_hat(1e-5)
    hxxy = (c[:, 0] ** 2 - THETA) * c[:, 1]
    assert abs((rr - bgk) @ hxxy) > 1e-9
    assert abs(rr.sum() - bgk.sum()) < TOL


@pytest.mark.parametrize("seed", range(3))
def test_trapezoidal_reconstruction(orc, seed):
    """App. F.5: with tau = nu/theta, tau_s = nu_t/theta and the unshifted CE part
    F1 = (tau/tau_hat) f1, the collision Q = f_post - f of the operational rule
    solves  Q = -F1/tau - (f + Q/2 - f0 - F1)/tau_s  (Eq. correct_Qi with the
    inverse shift substituted)."""
    q = 27
    f, S, rho, u = _state(orc, q, seed)
    nu, c_nu = 1e-5, 0.02
    f0, f1, fsgs, om_s = orc.closure_parts(q, CLOSURES["kcrb_h"], f, S, nu, c_nu)
    om = orc.omega_hat(nu)
    assert om_s < om
    fpost, _ = orc.collide_cell(q, CLOSURES["kcrb_h"], f, S, nu, c_nu)
    Q = fpost - f
    tau, tau_hat = nu / THETA, 1.0 / om
    tau_s = 1.0 / om_s - 0.5
    F1 = tau / tau_hat * f1
    rhs = -F1 / tau - (f + Q / 2 - f0 - F1) / tau_s
    # the relation divides O(1) populations by tau_s: round-off scales with |f|/tau_s
    assert np.abs(Q - rhs).max() < TOL * np.abs(f).max() / tau_s


def test_rate_formula(orc):
    nu = 1.59155e-4
    om = orc.omega_hat(nu)
    assert om == 1.0 / (3.0 * nu + 0.5)
    assert orc.omega_sgs(0.0, nu, 0.035) == om
    assert orc.omega_sgs(1e-12, nu, 0.035) == om  # clipped: C sqrt(k) < nu
    c_nu = 0.035
    trs = np.logspace(-8, -1, 30)
    vals = np.array([orc.omega_sgs(t, nu, c_nu) for t in trs])
    assert np.all(np.diff(vals) <= 0) and np.all(vals <= om)
    for t, v in zip(trs, vals):
        nut = c_nu * np.sqrt(abs(t) / 2.0)
        expect = om if nut <= nu else 1.0 / (3.0 * nut + 0.5)
        assert v == pytest.approx(expect, rel=1e-15)
    # the trace enters through its magnitude
    assert orc.omega_sgs(-1e-3, nu, c_nu) == orc.omega_sgs(1e-3, nu, c_nu)


def _rr_closed_form(axes, u, a2):
    """Recursive-regularised non-equilibrium coefficient of a mode given by its
    list of axes, in the closed form the recursion of Eq. (kcrr_rr) sums to in
    the isothermal case: the sum over all pairs (i, j) of the mode's indices of
    a2[a_i][a_j] times the product of u over the remaining indices (induction
    on n: the recursion's u_{a_n} term carries the pairs among the first n-1
    indices, its sum term the pairs (i, n))."""
    n = len(axes)
    s = 0.0
    for i in range(n):
        for j in range(i + 1, n):
            p = 1.0
            for k in range(n):
                if k != i and k != j:
                    p *= u[axes[k]]
            s += a2[axes[i]][axes[j]] * p
    return s


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("with_high_sgs", [False, True])
def test_kcrr_against_hermite_closed_form(orc, seed, with_high_sgs):
    """KC-RR (App. F.4) on a state built from its D3Q27 Hermite coefficients.

    The state is f = f0 + w sum_d N_d H_d K_d over the modes d of order >= 2,
    with H_d(c) = prod_a h(c_a, d_a), h = 1, c, c^2 - theta and N_d the
    quadrature normalisation prod_a (1, 1/theta, 1/(2 theta^2))[d_a] (the
    three-point rule per axis makes the 27 H_d orthogonal, so f's
    non-equilibrium coefficients are exactly K_d): second order
    K = m_CE + M_sgs, the 17 high-order modes K = a_rr (closed form above,
    seeded by m_CE = -2 rho theta tau_hat S) plus, optionally, a random SGS
    departure A.  KC-RR must return f0 + w sum_d N_d H_d K'_d with
    K' = (1 - omega) m_CE + (1 - omega_s) M_sgs and (1 - omega) a_rr +
    (1 - omega_s) A, omega_s from the rate formula on tr M_sgs.  A wrong index,
    a dropped term of the recursion or a wrong mode normalisation relaxes part
    of a coefficient at omega_s instead of omega (or rebuilds it wrongly),
    which this state shows at (omega - omega_s) of that part."""
    q = 27
    rng = np.random.default_rng(100 + seed)
    c, w, _ = orc.lattice(q)
    c = c.astype(int)
    rho = 1.0 + 0.05 * rng.standard_normal()
    u = 0.08 * rng.standard_normal(3)
    # product-form equilibrium written out (Sec. 7 / App. E)
    f0 = np.array([w[i] * rho * np.prod([1 + c[i, a] * u[a] / THETA + (c[i, a] ** 2 - THETA) * u[a] ** 2
                                         / (2 * THETA ** 2) for a in range(3)]) for i in range(q)])
    nu, c_nu = 1e-5, 0.5
    om = 1.0 / (nu / THETA + 0.5)
    tau_hat = 1.0 / om
    B = 0.01 * rng.standard_normal((3, 3))
    S = 0.5 * (B + B.T)
    mce = -2.0 * rho * THETA * tau_hat * S
    C = 0.004 * rng.standard_normal((3, 3))
    Msgs = 0.5 * (C + C.T) + 0.004 * np.eye(3)
    tr = np.trace(Msgs)
    nut = c_nu * np.sqrt(abs(tr) / 2.0)
    assert nut > nu
    om_s = 1.0 / (nut / THETA + 0.5)
    assert om - om_s > 0.1

    def h(ci, d):
        return 1.0 if d == 0 else (float(ci) if d == 1 else ci * ci - THETA)

    norm = (1.0, 1.0 / THETA, 1.0 / (2.0 * THETA ** 2))
    modes = [(dx, dy, dz) for dz in range(3) for dy in range(3) for dx in range(3) if dx + dy + dz >= 2]
    K, Kp = {}, {}
    for d in modes:
        axes = [a for a in range(3) for _ in range(d[a])]
        if len(axes) == 2:
            i, j = axes
            K[d] = mce[i, j] + Msgs[i, j]
            Kp[d] = (1 - om) * mce[i, j] + (1 - om_s) * Msgs[i, j]
        else:
            arr = _rr_closed_form(axes, u, mce)
            A = 1e-3 * rng.standard_normal() if with_high_sgs else 0.0
            K[d] = arr + A
            Kp[d] = (1 - om) * arr + (1 - om_s) * A

    def build(coef):
        g = np.zeros(q)
        for i in range(q):
            for d, k in coef.items():
                g[i] += k * np.prod([norm[d[a]] * h(c[i, a], d[a]) for a in range(3)])
        return w * g

    f = f0 + build(K)
    expect = f0 + build(Kp)
    fpost, om_s_orc = orc.collide_cell(q, CLOSURES["kcrr"], f, S, nu, c_nu)
    assert om_s_orc == pytest.approx(om_s, rel=1e-12)
    scale = np.abs(expect - f0).max()
    assert np.abs(fpost - expect).max() <= 1e-12 * scale + 64 * EPS
