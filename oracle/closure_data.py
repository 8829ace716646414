"""FP64 oracle of the learned closure's training data (test infrastructure only).

Targets come from fine-lattice runs box-filtered to the coarse grid:
  - filtered populations  f_bar = box average of the fine populations over
    F^3 fine cells (the coarse LES state);
  - filtered density rho_bar = sum f_bar, Favre velocity u~ = sum f_bar c / rho_bar;
  - exact SGS stress, Eq. (m_sgs_2):  m_sgs = rho_bar (u u~ - u~ u~)
        = bar(rho u u) - bar(rho u) bar(rho u) / rho_bar,
    with rho, u the fine cells' moments (App. F.1 step 1).
Inputs of the network, per coarse cell (App. F.3 quantities of the coarse state):
  x[0:6]  m_neq / rho_bar, m_neq = sum (f_bar - f0(rho_bar, u~)) c c   (xx, yy, zz, xy, xz, yz)
  x[6:9]  invariants of A = m_CE / rho_bar = -2 theta tau_hat S (trace, second
          invariant (tr^2 - tr A^2)/2, determinant), S from the coarse u~ with the
          central differences of Eq. (fd) (periodic)
  x[9]    tau_hat = nu_c/theta + 1/2 of the coarse lattice
Target: m_sgs / rho_bar (same component order).
Under acoustic scaling (same lattice speed) the coarse viscosity in coarse
lattice units is nu_fine / F.

Plain numpy (the equilibrium comes from the C oracle), written for checking by eye.
"""
from __future__ import annotations

import numpy as np

import oracle

COMP = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def box_filter(a: np.ndarray, F: int) -> np.ndarray:
    """Average over F^3 blocks of the last three axes (z, y, x)."""
    *lead, nz, ny, nx = a.shape
    b = a.reshape(*lead, nz // F, F, ny // F, F, nx // F, F)
    return b.mean(axis=(-5, -3, -1))


def stream(f: np.ndarray) -> np.ndarray:
    """Periodic pull streaming, Eq. (streaming): f_i(x) <- f_i(x - c_i)."""
    c, _, _ = oracle.lattice(f.shape[0])
    return np.stack([np.roll(f[i], shift=(c[i, 2], c[i, 1], c[i, 0]), axis=(0, 1, 2)) for i in range(f.shape[0])])


def filtered_state(f_fine: np.ndarray, F: int, neq_scale: float = 1.0, pull: bool = False):
    """(f_bar [q, nz/F, ny/F, nx/F], m_sgs [6, ...]) from fine populations f_fine [q, nz, ny, nx].

    With neq_scale r != 1 the non-equilibrium part of the fine populations is
    rescaled before filtering, f_bar = bar(f) + (r - 1) bar(f - f0(rho, u)) with
    f0 each fine cell's own equilibrium: under acoustic scaling (dt_c = F dt_f)
    the coarse lattice's first-order non-equilibrium part of the same flow is
    r = F tau_hat_c / tau_hat_f times the filtered fine one (f1 ~ tau_hat S dt),
    while the SGS part bar(f0) - f0(rho_bar, u_bar) (Eq. fsgs_def) is kept.
    With pull, the streamed populations (the pre-collision state of the next
    step, from which a step computes its closure inputs) are filtered."""
    if pull:
        f_fine = stream(f_fine)
    q = f_fine.shape[0]
    c, _, _ = oracle.lattice(q)
    rho = f_fine.sum(axis=0)
    mom = np.einsum("iabc,ik->kabc", f_fine, c.astype(float))
    u = mom / rho
    f_bar = box_filter(f_fine, F)
    if neq_scale != 1.0:
        f_bar = f_bar + (neq_scale - 1.0) * box_filter(f_fine - oracle.init_equilibrium(q, rho, u), F)
    rho_bar = box_filter(rho, F)
    rhou_bar = box_filter(mom, F)
    msgs = np.empty((6,) + rho_bar.shape)
    for k, (a, b) in enumerate(COMP):
        msgs[k] = box_filter(rho * u[a] * u[b], F) - rhou_bar[a] * rhou_bar[b] / rho_bar
    return f_bar, msgs


def features(f_bar: np.ndarray, nu_coarse: float):
    """Network inputs x [n, 10] and rho_bar [n] of every coarse cell (x fastest)."""
    q = f_bar.shape[0]
    c, _, _ = oracle.lattice(q)
    cf = c.astype(float)
    rho, u = oracle.fields(f_bar)
    f0 = oracle.init_equilibrium(q, rho, u)
    mneq = np.einsum("iabc,ik,il->klabc", f_bar - f0, cf, cf)
    S = oracle.strain_field(u)
    tau_hat = nu_coarse / oracle.THETA + 0.5
    A = -2.0 * oracle.THETA * tau_hat * S  # m_CE / rho
    n = rho.size
    x = np.empty((n, 10))
    # the KC-MP carrier (m_neq - m_CE)/rho (App. F.3): the non-equilibrium second
    # moment beyond its Chapman-Enskog part
    for k, (a, b) in enumerate(COMP):
        x[:, k] = (mneq[a, b] / rho - A[a, b]).ravel()
    Am = np.moveaxis(A.reshape(3, 3, n), 2, 0)  # [n, 3, 3]
    tr = np.trace(Am, axis1=1, axis2=2)
    tr2 = np.einsum("nab,nba->n", Am, Am)
    x[:, 6] = tr
    x[:, 7] = 0.5 * (tr * tr - tr2)
    x[:, 8] = np.linalg.det(Am)
    x[:, 9] = tau_hat
    return x, rho.ravel()


def targets(msgs: np.ndarray, rho_bar: np.ndarray) -> np.ndarray:
    """m_sgs / rho_bar as [n, 6]."""
    return (msgs.reshape(6, -1) / rho_bar.reshape(1, -1)).T.copy()
