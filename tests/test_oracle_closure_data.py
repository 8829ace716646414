"""Pins of the learned closure's training-data oracle (no GPU):
  - box filter of a constant and of a linear field;
  - Eq. (m_sgs_2): for a fine state that is uniform inside every filter box
    the exact SGS stress vanishes; for two-valued velocity inside a box it equals
    the textbook covariance rho_bar (<u u> - <u><u>) (equal densities), and with
    two densities the density-weighted covariance of two parcels;
  - the carrier inputs (m_neq - m_CE)/rho of an equilibrium state are
    2 theta tau_hat S; an added second-order Hermite mode moves only its own
    component, by the mode's coefficient;
  - the strain invariants of a pure shear field;
  - the rescaled non-equilibrium part of the consistent coarse state: no effect
    on an equilibrium state, exactly r times an added zero-mass, zero-momentum
    Hermite mode, and mass and momentum of any state unchanged."""
import numpy as np
import pytest

import oracle
from oracle import closure_data as cd
from paper_2605_19796_gb300 import inputs


def test_box_filter():
    a = np.arange(8 * 8 * 8, dtype=float).reshape(8, 8, 8)
    b = cd.box_filter(a, 4)
    assert b.shape == (2, 2, 2)
    assert b[0, 0, 0] == pytest.approx(a[:4, :4, :4].mean())
    assert np.allclose(cd.box_filter(np.full((2, 8, 8, 8), 3.0), 2), 3.0)


def test_msgs_zero_for_box_uniform_state():
    rho_c, u_c = inputs.hit_fields(4, k0=1.0, urms=0.05, seed=1)
    u = np.repeat(np.repeat(np.repeat(u_c, 2, axis=1), 2, axis=2), 2, axis=3)
    f = oracle.init_equilibrium(27, None, u)
    _, msgs = cd.filtered_state(f, 2)
    assert np.abs(msgs).max() < 1e-16


def test_msgs_two_valued_velocity_covariance():
    """Inside each 2^3 box half the cells move with u1, half with u2 (rho = 1):
    m_sgs = (<uu> - <u><u>) = (u1 - u2)(u1 - u2)^T / 4."""
    u = np.zeros((3, 4, 4, 4))
    u1, u2 = np.array([0.03, -0.01, 0.02]), np.array([-0.02, 0.015, 0.0])
    for a in range(3):
        u[a, :, :, 0::2] = u1[a]
        u[a, :, :, 1::2] = u2[a]
    f = oracle.init_equilibrium(27, None, u)
    _, msgs = cd.filtered_state(f, 2)
    d = u1 - u2
    for k, (a, b) in enumerate(cd.COMP):
        assert np.allclose(msgs[k], d[a] * d[b] / 4, rtol=1e-12, atol=1e-17)


def test_msgs_two_valued_density_and_velocity():
    """Half the cells of each 2^3 box hold (rho1, u1), half (rho2, u2): Eq.
    (m_sgs_2) gives bar(rho u u) - bar(rho u) bar(rho u) / bar(rho) =
    rho1 rho2 / (2 (rho1 + rho2)) (u1 - u2)(u1 - u2)^T, the density-weighted
    covariance of two equal parcels."""
    u = np.zeros((3, 4, 4, 4))
    rho = np.zeros((4, 4, 4))
    u1, u2 = np.array([0.03, -0.01, 0.02]), np.array([-0.02, 0.015, 0.0])
    r1, r2 = 1.1, 0.95
    rho[:, 0::2, :], rho[:, 1::2, :] = r1, r2
    for a in range(3):
        u[a, :, 0::2, :] = u1[a]
        u[a, :, 1::2, :] = u2[a]
    f = oracle.init_equilibrium(27, rho, u)
    _, msgs = cd.filtered_state(f, 2)
    d = u1 - u2
    for k, (a, b) in enumerate(cd.COMP):
        assert np.allclose(msgs[k], r1 * r2 / (2 * (r1 + r2)) * d[a] * d[b], rtol=1e-11, atol=1e-17)


def test_features_equilibrium_and_hermite_mode():
    rho, u = inputs.hit_fields(6, k0=1.0, urms=0.04, seed=2)
    f = oracle.init_equilibrium(27, rho, u)
    x, r = cd.features(f, 1e-4)
    # no non-equilibrium part: the carrier inputs are -m_CE/rho = 2 theta tau_hat S
    S = oracle.strain_field(u)
    tau_hat = 1e-4 * 3 + 0.5
    for k, (a, b) in enumerate(cd.COMP):
        ref = (2 * oracle.THETA * tau_hat * S[a, b]).ravel()
        assert np.abs(x[:, k] - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.allclose(x[:, 9], tau_hat)
    c, w, _ = oracle.lattice(27)
    cf = c.astype(float)
    amp = 1e-4
    Hxy = (w * cf[:, 0] * cf[:, 1])[:, None, None, None]
    g = f + amp * Hxy / oracle.THETA ** 2
    x2, r2 = cd.features(g, 1e-4)
    # the mode carries no mass or momentum: only the xy carrier input moves, by amp/rho
    assert np.allclose(x2[:, 3] - x[:, 3], amp / r2, rtol=1e-9)
    assert np.abs(x2[:, [0, 1, 2, 4, 5]] - x[:, [0, 1, 2, 4, 5]]).max() < 1e-15
    assert np.abs(x2[:, 6:] - x[:, 6:]).max() <= 1e-12 * np.abs(x[:, 6:]).max()


def test_strain_invariants_of_pure_shear():
    n = 8
    u = np.zeros((3, n, n, n))
    y = np.arange(n)
    u[0] = (0.01 * np.sin(2 * np.pi * y / n))[None, :, None]
    f = oracle.init_equilibrium(27, None, u)
    x, _ = cd.features(f, 1e-3)
    tau = 1e-3 * 3 + 0.5
    S = oracle.strain_field(u)
    sxy = S[0, 1].ravel()
    assert np.abs(x[:, 6]).max() < 1e-15                                         # trace
    assert np.allclose(x[:, 7], -(2 * oracle.THETA * tau) ** 2 * sxy ** 2, atol=1e-18)  # -A_xy^2
    assert np.abs(x[:, 8]).max() < 1e-18                                          # det


@pytest.mark.parametrize("q", [19, 27])
def test_neq_rescale_equilibrium_state_unchanged(q):
    rho, u = inputs.hit_fields(8, k0=2.0, urms=0.05, seed=6)
    f = oracle.init_equilibrium(q, rho, u)
    a, ma = cd.filtered_state(f, 2)
    b, mb = cd.filtered_state(f, 2, neq_scale=3.7)
    assert np.abs(a - b).max() < 1e-15 and np.array_equal(ma, mb)


@pytest.mark.parametrize("q", [19, 27])
def test_neq_rescale_scales_an_added_hermite_mode(q):
    """delta_i = w_i c_ix c_iy eps(x) carries no mass and no momentum, so it is
    exactly the non-equilibrium part f - f0(rho, u) of f0 + delta."""
    c, w, _ = oracle.lattice(q)
    rho, u = inputs.hit_fields(8, k0=2.0, urms=0.05, seed=7)
    f0 = oracle.init_equilibrium(q, rho, u)
    eps = np.random.default_rng(3).standard_normal((8, 8, 8)) * 1e-3
    delta = (w * c[:, 0] * c[:, 1])[:, None, None, None] * eps[None]
    r = 3.7
    got, _ = cd.filtered_state(f0 + delta, 2, neq_scale=r)
    ref = cd.box_filter(f0, 2) + r * cd.box_filter(delta, 2)
    assert np.abs(got - ref).max() < 1e-15


def test_neq_rescale_keeps_mass_and_momentum():
    rng = np.random.default_rng(9)
    c, w, _ = oracle.lattice(27)
    f = w[:, None, None, None] * (1 + 0.05 * rng.standard_normal((27, 8, 8, 8)))
    a, _ = cd.filtered_state(f, 4)
    b, _ = cd.filtered_state(f, 4, neq_scale=0.25)
    assert np.abs(a.sum(0) - b.sum(0)).max() < 1e-15
    cf = c.astype(float)
    assert np.abs(np.einsum("iabc,ik->kabc", a - b, cf)).max() < 1e-15


@pytest.mark.parametrize("q", [19, 27])
def test_pull_filters_the_streamed_state(q):
    """The pulled state equals one step of the C oracle with no relaxation
    (BGK at nu -> infinity: omega -> 0, the step is pure streaming)."""
    rng = np.random.default_rng(11)
    c, w, _ = oracle.lattice(q)
    f = w[:, None, None, None] * (1 + 0.05 * rng.standard_normal((q, 8, 8, 8)))
    ref = oracle.run(f, 1, closure=0, nu=1e15)
    a, ma = cd.filtered_state(f, 2, pull=True)
    b, mb = cd.filtered_state(ref, 2)
    assert np.abs(a - b).max() < 1e-14 and np.abs(ma - mb).max() < 1e-14
