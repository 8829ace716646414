"""Pins of the oracle's lattice tables and equilibrium against the paper and
against mathematics (no GPU).

Lattice: App. F "Velocity space discretization" (D3Q27 as the Cartesian
product of D1Q3 with weights 2/3 and 1/6, theta_R = 1/3); D3Q19 is the
textbook lattice (weights 1/3, 1/18, 1/36).  Equilibrium: Eq.
(discrete_equilibrium) and the moment relations of App. F ("Macroscopic fields
and isothermal discrete equilibrium") and App. E.
"""
import itertools

import numpy as np
import pytest

THETA = 1.0 / 3.0


def _d1q3_weight(c):
    return 2.0 / 3.0 if c == 0 else 1.0 / 6.0


@pytest.mark.parametrize("q", [19, 27])
def test_canonical_order_and_opposites(orc, q):
    c, w, opp = orc.lattice(q)
    expect = [v for v in itertools.product((-1, 0, 1), repeat=3)]  # (cz, cy, cx), cx fastest
    expect = [(cx, cy, cz) for (cz, cy, cx) in expect if not (q == 19 and abs(cx) + abs(cy) + abs(cz) == 3)]
    assert [tuple(r) for r in c] == expect
    for i in range(q):
        assert tuple(c[opp[i]]) == tuple(-c[i])
        assert opp[opp[i]] == i


def test_d3q27_weights_are_d1q3_products(orc):
    c, w, _ = orc.lattice(27)
    for i in range(27):
        assert w[i] == pytest.approx(np.prod([_d1q3_weight(x) for x in c[i]]), abs=1e-17)
    # the four distinct values
    assert sorted(set(np.round(w, 15))) == sorted(np.round([8 / 27, 2 / 27, 1 / 54, 1 / 216], 15))


def test_d3q19_weights_textbook(orc):
    c, w, _ = orc.lattice(19)
    s = np.abs(c).sum(axis=1)
    assert np.allclose(w[s == 0], 1 / 3) and np.allclose(w[s == 1], 1 / 18) and np.allclose(w[s == 2], 1 / 36)
    assert (s == 1).sum() == 6 and (s == 2).sum() == 12


@pytest.mark.parametrize("q", [19, 27])
def test_quadrature_isotropy(orc, q):
    """sum w = 1, sum w c = 0, sum w cc = theta delta, odd moments vanish,
    sum w c_a c_b c_c c_d = theta^2 (d_ab d_cd + d_ac d_bd + d_ad d_bc)."""
    c, w, _ = orc.lattice(q)
    c = c.astype(float)
    d = np.eye(3)
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.abs(np.einsum("i,ia->a", w, c)).max() < 1e-16
    assert np.abs(np.einsum("i,ia,ib->ab", w, c, c) - THETA * d).max() < 1e-16
    assert np.abs(np.einsum("i,ia,ib,ic->abc", w, c, c, c)).max() < 1e-16
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    iso = THETA ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                        + np.einsum("ad,bc->abcd", d, d))
    assert np.abs(m4 - iso).max() < 1e-16


def test_d3q27_aliasing(orc):
    """On D3Q27, c^3 = c (App. F: directional powers above two alias)."""
    c, _, _ = orc.lattice(27)
    assert np.array_equal(c ** 3, c) and np.array_equal(c ** 4, c ** 2)


def _rand_state(seed):
    rng = np.random.default_rng(seed)
    return 1.0 + 0.1 * rng.standard_normal(), 0.15 * rng.standard_normal(3)


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("seed", range(5))
def test_equilibrium_moments(orc, q, seed):
    """sum f0 = rho, sum f0 c = rho u, sum f0 cc = rho (uu + theta delta) (App. E, App. F)."""
    rho, u = _rand_state(seed)
    c, _, _ = orc.lattice(q)
    c = c.astype(float)
    f0 = orc.equilibrium(q, rho, u)
    assert f0.sum() == pytest.approx(rho, rel=1e-15)
    assert np.abs(f0 @ c - rho * u).max() < 1e-15
    m2 = np.einsum("i,ia,ib->ab", f0, c, c)
    assert np.abs(m2 - rho * (np.outer(u, u) + THETA * np.eye(3))).max() < 1e-15


@pytest.mark.parametrize("seed", range(5))
def test_d3q27_product_form_closed_form(orc, seed):
    """Eq. (discrete_equilibrium) restated through the known closed form of the
    D1Q3 factor: psi(0,u) = 2/3 - u^2, psi(+-1,u) = (1/3 + u^2 +- u)/2, so that
    f0_i = rho prod_a psi(c_ia, u_a).  Also the tensor-product moments
    sum f0 cx^2 cy = rho u_y (theta + ux^2) and sum f0 cx^2 cy^2 cz^2 = rho prod (theta + u_a^2)."""
    rho, u = _rand_state(seed)
    c, _, _ = orc.lattice(27)
    f0 = orc.equilibrium(27, rho, u)

    def psi(ci, ua):
        return 2.0 / 3.0 - ua * ua if ci == 0 else (1.0 / 3.0 + ua * ua + ci * ua) / 2.0

    ref = np.array([rho * psi(ci[0], u[0]) * psi(ci[1], u[1]) * psi(ci[2], u[2]) for ci in c])
    assert np.abs(f0 - ref).max() < 2e-16
    cf = c.astype(float)
    assert (f0 * cf[:, 0] ** 2 * cf[:, 1]).sum() == pytest.approx(rho * u[1] * (THETA + u[0] ** 2), rel=1e-13)
    assert (f0 * (cf ** 2).prod(axis=1)).sum() == pytest.approx(rho * np.prod(THETA + u ** 2), rel=1e-14)


@pytest.mark.parametrize("q", [19, 27])
def test_equilibrium_at_rest_is_weights(orc, q):
    _, w, _ = orc.lattice(q)
    assert np.abs(orc.equilibrium(q, 1.3, [0.0, 0.0, 0.0]) - 1.3 * w).max() < 1e-16


def test_d3q19_equilibrium_second_order_hermite(orc):
    """Reading for D3Q19: w rho (1 + c.u/theta + (c.u)^2/(2 theta^2) - u^2/(2 theta)),
    checked on the textbook values 1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u^2."""
    rho, u = 0.97, np.array([0.05, -0.02, 0.03])
    c, w, _ = orc.lattice(19)
    cu = c @ u
    ref = w * rho * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * u @ u)
    assert np.abs(orc.equilibrium(19, rho, u) - ref).max() < 1e-16
