"""FP64 oracle of one learned-closure time step (test infrastructure only).

The learned closure is KC-MP (App. F.3) with the SGS second moment taken from
the network instead of m_neq - m_CE:
  1. pull streaming, Eq. (streaming); rho, u (App. F.1 step 1); f0 (Eq. discrete_equilibrium)
  2. strain S (Eqs. fd, strain_rate_discrete)
  3. inputs x: the KC-MP carrier (m_neq - m_CE) / rho (6), trace / second
     invariant / determinant of m_CE / rho = -2 theta tau_hat S (3), tau_hat (1);
     standardised
  4. network (oracle/mlp.py) -> standardised m_sgs / rho -> m_sgs
  5. k = |tr m_sgs| / 2, omega_s (Eq. omega_sgs_operational)
  6. f_post = f - omega (f - f0 - f_sgs) - omega_s f_sgs, f_sgs = w/(2 theta^2) H : m_sgs

Precision: the CUDA kernel evaluates the network on BF16 tensor cores (BF16
inputs, weights and hidden activations, FP32 accumulation).  With
``bf16=True`` this oracle rounds the same quantities to BF16
(round-to-nearest-even, emulated on float32 bit patterns) and accumulates in
FP64, so both sides take the BF16 rounding decisions at the same points.
"""
from __future__ import annotations

import numpy as np

import oracle
from oracle import mlp

THETA = oracle.THETA
COMP = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def bf16(a: np.ndarray) -> np.ndarray:
    """Round to bfloat16 (nearest, ties to even) and return as float64."""
    x = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (x >> 16) & 1
    r = ((x + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(params_flat: np.ndarray, xs: np.ndarray, rounding: bool):
    p = mlp.unflat(np.asarray(params_flat, dtype=np.float64))
    if not rounding:
        ys, _ = mlp.forward(p, xs)
        return ys
    h = bf16(xs)
    for l in range(1, 4):
        a = h @ bf16(p[f"W{l}"]).T + p[f"b{l}"]
        h = bf16(mlp.silu(a))
    return h @ bf16(p["W4"]).T + p["b4"]


def inputs_and_state(f_post_prev: np.ndarray, nu: float):
    """Streamed populations, rho, u, f0, network inputs x [N, 10] (pre-standardisation)."""
    q = f_post_prev.shape[0]
    c, w, _ = oracle.lattice(q)
    fp = np.empty_like(f_post_prev)
    for i in range(q):
        fp[i] = np.roll(f_post_prev[i], shift=(c[i, 2], c[i, 1], c[i, 0]), axis=(0, 1, 2))
    rho, u = oracle.fields(fp)
    f0 = oracle.init_equilibrium(q, rho, u)
    cf = c.astype(float)
    mneq = np.einsum("iabc,ik,il->klabc", fp - f0, cf, cf)
    S = oracle.strain_field(u)
    tau_hat = nu / THETA + 0.5
    A = -2.0 * THETA * tau_hat * S
    n = rho.size
    x = np.empty((n, 10))
    for k, (a, b) in enumerate(COMP):
        x[:, k] = (mneq[a, b] / rho - A[a, b]).ravel()
    Am = np.moveaxis(A.reshape(3, 3, n), 2, 0)
    tr = np.trace(Am, axis1=1, axis2=2)
    x[:, 6] = tr
    x[:, 7] = 0.5 * (tr * tr - np.einsum("nab,nba->n", Am, Am))
    x[:, 8] = np.linalg.det(Am)
    x[:, 9] = tau_hat
    return fp, rho, u, f0, x


def step(f: np.ndarray, nu: float, params: np.ndarray, stats: np.ndarray, c_nu: float, delta: float = 1.0,
         rounding: bool = True):
    """One learned-closure step of a periodic box; returns (f_post, m_sgs [N, 6])."""
    q = f.shape[0]
    c, w, _ = oracle.lattice(q)
    cf = c.astype(float)
    fp, rho, u, f0, x = inputs_and_state(f, nu)
    stats = np.asarray(stats, dtype=np.float64)
    xmu, xsd, ymu, ysd = stats[:10], stats[10:20], stats[20:26], stats[26:32]
    xs = (x - xmu) / xsd
    ys = forward(params, xs, rounding)
    r = rho.ravel()
    msgs = r[:, None] * (ys * ysd + ymu)
    omega = oracle.omega_hat(nu)
    tr = msgs[:, 0] + msgs[:, 1] + msgs[:, 2]
    nut = c_nu * delta * np.sqrt(np.abs(tr) / 2.0)
    omega_s = np.where(nut > nu, 1.0 / (nut / THETA + 0.5), omega)
    M = np.zeros((3, 3, r.size))
    for k, (a, b) in enumerate(COMP):
        M[a, b] = msgs[:, k]
        M[b, a] = msgs[:, k]
    shp = f.shape[1:]
    hm = np.einsum("ia,ib,abn->in", cf, cf, M) - THETA * tr[None, :]
    fsgs = (w[:, None] / (2 * THETA ** 2) * hm).reshape((q,) + shp)
    fpost = fp - omega * (fp - f0 - fsgs) - omega_s.reshape(shp)[None] * fsgs
    return fpost, msgs
