"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module holds initial conditions only (density and velocity fields, or
random populations for identity checks); it contains none of the lattice
method's arithmetic and imports nothing else from this package, so both the
CUDA-path tests and the oracle may use it.

Fields are FP64 numpy arrays: ``rho[nz, ny, nx]`` and ``u[3, nz, ny, nx]``,
x fastest, lattice units.
"""
from __future__ import annotations

import math
from typing import Optional, Tuple

import numpy as np

THETA_LATTICE = 1.0 / 3.0  # c_s^2 of the D3Q19/D3Q27 lattices (Sec. 7 / App. F)


def tgv_fields(n: int, u0: float = 0.05, rho0: float = 1.0,
               shape: Optional[Tuple[int, int, int]] = None) -> Tuple[np.ndarray, np.ndarray]:
    """Taylor-Green vortex initial state (Sec. 7.1).

    u_x = u0 sin X cos Y cos Z, u_y = -u0 cos X sin Y cos Z, u_z = 0 with
    X = 2 pi x / L_box (node positions x = 0..n-1).  The pressure fluctuation
    p = rho0 u0^2/16 (cos 2X + cos 2Y)(cos 2Z + 2) enters as rho = rho0 + p/theta.
    """
    nx, ny, nz = shape if shape is not None else (n, n, n)
    X = 2.0 * math.pi * np.arange(nx) / nx
    Y = 2.0 * math.pi * np.arange(ny) / ny
    Z = 2.0 * math.pi * np.arange(nz) / nz
    Zg, Yg, Xg = np.meshgrid(Z, Y, X, indexing="ij")
    u = np.zeros((3, nz, ny, nx), dtype=np.float64)
    u[0] = u0 * np.sin(Xg) * np.cos(Yg) * np.cos(Zg)
    u[1] = -u0 * np.cos(Xg) * np.sin(Yg) * np.cos(Zg)
    p = rho0 * u0 * u0 / 16.0 * (np.cos(2 * Xg) + np.cos(2 * Yg)) * (np.cos(2 * Zg) + 2.0)
    rho = rho0 + p / THETA_LATTICE
    return rho, u


def tgv2d_fields(n: int, u0: float = 0.01, nz: int = 4) -> Tuple[np.ndarray, np.ndarray]:
    """Two-dimensional Taylor-Green vortex, uniform in z (an exact Navier-Stokes
    solution whose kinetic energy decays as exp(-2 nu |k|^2 t), |k|^2 = 2 (2 pi/n)^2).
    rho carries the exact pressure p = -rho0 u0^2/4 (cos 2X + cos 2Y)."""
    X = 2.0 * math.pi * np.arange(n) / n
    Yg, Xg = np.meshgrid(X, X, indexing="ij")
    u = np.zeros((3, nz, n, n), dtype=np.float64)
    u[0] = (u0 * np.sin(Xg) * np.cos(Yg))[None]
    u[1] = (-u0 * np.cos(Xg) * np.sin(Yg))[None]
    p = -u0 * u0 / 4.0 * (np.cos(2 * Xg) + np.cos(2 * Yg))
    rho = np.broadcast_to(1.0 + p / THETA_LATTICE, (nz, n, n)).copy()
    return rho, u


def shear_wave_fields(n: int, amp: float = 1e-3, nxy: int = 4) -> Tuple[np.ndarray, np.ndarray]:
    """u_x = amp sin(2 pi z / n), uniform in x and y, rho = 1 (decays as exp(-nu k^2 t))."""
    z = np.arange(n)
    u = np.zeros((3, n, nxy, nxy), dtype=np.float64)
    u[0] = (amp * np.sin(2.0 * math.pi * z / n))[:, None, None]
    rho = np.ones((n, nxy, nxy), dtype=np.float64)
    return rho, u


def _hit_low_modes(shape, k0: float, seed: int):
    """Seeded solenoidal low-mode block of the HIT spectrum.

    Only |k_a| <= kmax_a = min(6 k0, (n_a - 1)//2) carry energy (E(6 k0) / E(k0)
    ~ 1e-27).  Returns (block[3, 2kz+1, 2ky+1, kx+1] complex128, (kmx, kmy, kmz)).
    """
    nx, ny, nz = shape
    kc = int(math.ceil(6.0 * k0))
    kmx, kmy, kmz = (min(kc, (n - 1) // 2) for n in (nx, ny, nz))
    rng = np.random.Generator(np.random.PCG64(seed))
    kx = np.arange(0, kmx + 1, dtype=np.float64)
    ky = np.arange(-kmy, kmy + 1, dtype=np.float64)
    kz = np.arange(-kmz, kmz + 1, dtype=np.float64)
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    k2 = KX * KX + KY * KY + KZ * KZ
    k = np.sqrt(k2)
    with np.errstate(divide="ignore", invalid="ignore"):
        amp = np.where(k > 0, np.sqrt(k ** 4 * np.exp(-2.0 * (k / k0) ** 2) / (4.0 * math.pi * k2)), 0.0)
    blk = np.empty((3,) + k.shape, dtype=np.complex128)
    for a in range(3):
        blk[a] = (rng.standard_normal(k.shape) + 1j * rng.standard_normal(k.shape)) * amp
    with np.errstate(divide="ignore", invalid="ignore"):
        kdotu = (KX * blk[0] + KY * blk[1] + KZ * blk[2]) / np.where(k2 > 0, k2, 1.0)
    blk[0] -= KX * kdotu
    blk[1] -= KY * kdotu
    blk[2] -= KZ * kdotu
    return blk, (kmx, kmy, kmz)


def hit_fields(n: int, k0: float = 4.0, urms: float = 0.04, seed: int = 0,
               shape: Optional[Tuple[int, int, int]] = None, device=None):
    """Decaying homogeneous isotropic turbulence initial velocity.

    Random-phase solenoidal field with energy spectrum E(k) ~ k^4 exp(-2 (k/k0)^2),
    k in units of 2 pi / L.  Recipe: complex Gaussian noise from a seeded PCG64
    generator on the rfft half-spectrum modes |k_a| <= min(6 k0, (n_a-1)/2),
    times the amplitude sqrt(E(k) / (4 pi k^2)), projected onto the plane normal
    to k (u <- u - k (k.u)/k^2), inverse real FFT (Hermitian completion of the
    k_x = 0 plane by the transform), zero mean, then rescaled so that the
    per-component rms sqrt(<u_a^2>) averaged over the three components equals
    ``urms``.  rho = 1.

    ``device=None`` returns numpy FP64 arrays (rho[nz,ny,nx], u[3,nz,ny,nx]);
    a torch device (e.g. "cuda") runs the inverse FFT there and returns torch
    FP64 tensors with the same values up to FFT rounding.
    """
    nx, ny, nz = shape if shape is not None else (n, n, n)
    blk, (kmx, kmy, kmz) = _hit_low_modes((nx, ny, nz), k0, seed)
    # block index -k..k maps to the FFT index (k mod n)
    zi = np.array([(k + nz) % nz for k in range(-kmz, kmz + 1)])
    yi = np.array([(k + ny) % ny for k in range(-kmy, kmy + 1)])
    if device is None:
        import scipy.fft as sfft

        u = np.empty((3, nz, ny, nx), dtype=np.float64)
        for a in range(3):
            spec = np.zeros((nz, ny, nx // 2 + 1), dtype=np.complex128)
            spec[np.ix_(zi, yi, np.arange(kmx + 1))] = blk[a]
            u[a] = sfft.irfftn(spec, s=(nz, ny, nx), workers=-1)
        u -= u.reshape(3, -1).mean(axis=1)[:, None, None, None]
        u *= urms / math.sqrt(float(np.mean(u * u)))
        return np.ones((nz, ny, nx), dtype=np.float64), u
    import torch

    u = torch.empty((3, nz, ny, nx), dtype=torch.float64, device=device)
    zt = torch.as_tensor(zi, device=device)
    yt = torch.as_tensor(yi, device=device)
    for a in range(3):
        spec = torch.zeros((nz, ny, nx // 2 + 1), dtype=torch.complex128, device=device)
        b = torch.as_tensor(blk[a], device=device)
        spec.index_put_((zt[:, None, None], yt[None, :, None], torch.arange(kmx + 1, device=device)[None, None, :]), b)
        u[a] = torch.fft.irfftn(spec, s=(nz, ny, nx))
        del spec
    u -= u.reshape(3, -1).mean(dim=1)[:, None, None, None]
    u *= urms / torch.sqrt(torch.mean(u * u))
    return torch.ones((nz, ny, nx), dtype=torch.float64, device=device), u


def channel_fields(nx: int, ny: int, nz: int, u_bulk: float, amp: float = 0.05, seed: int = 0,
                   device=None):
    """Plane channel between walls at y = -1/2 and y = ny - 1/2 (halfway bounce-back):
    laminar profile u_x = 1.5 u_bulk (1 - ((y - h)/h)^2), h = ny/2, y = j + 1/2,
    plus seeded divergence-free perturbations u' = curl(psi e_y-ish streamfunction),
    psi = amp u_bulk h sin^2(pi y/ny) sum of a few random Fourier modes in x and z.
    rho = 1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    y = (np.arange(ny) + 0.5)
    h = ny / 2.0
    base = 1.5 * u_bulk * (1.0 - ((y - h) / h) ** 2)
    X = 2 * math.pi * np.arange(nx) / nx
    Z = 2 * math.pi * np.arange(nz) / nz
    env = np.sin(math.pi * y / ny) ** 2
    denv = (2 * math.pi / ny) * np.sin(math.pi * y / ny) * np.cos(math.pi * y / ny)
    u = np.zeros((3, nz, ny, nx))
    u[0] += base[None, :, None]
    for _ in range(6):
        kx, kz = rng.integers(1, 5), rng.integers(1, 5)
        ph1, ph2 = rng.uniform(0, 2 * math.pi, 2)
        a = amp * u_bulk * rng.uniform(0.5, 1.0)
        # streamfunction psi(x,y) = a h env(y) sin(kx X + ph1) in the x-y plane: u = dpsi/dy, v = -dpsi/dx
        sx = np.sin(kx * X + ph1)[None, :]
        cx = np.cos(kx * X + ph1)[None, :]
        mod = np.cos(kz * Z + ph2)[:, None, None]
        u[0] += mod * (a * h * denv[:, None] * sx)[None]
        u[1] += mod * (-a * h * env[:, None] * cx * (2 * math.pi * kx / nx))[None]
    rho = np.ones((nz, ny, nx))
    if device is not None:
        import torch

        return torch.as_tensor(rho, device=device), torch.as_tensor(u, device=device)
    return rho, u


def random_populations(q: int, shape: Tuple[int, int, int], seed: int = 0, amp: float = 0.05,
                       weights: Optional[np.ndarray] = None) -> np.ndarray:
    """Random positive populations f[q, nz, ny, nx] = w_i (1 + amp * N(0,1)).

    ``weights`` are the lattice weights (passed in by the caller so that this
    module carries no lattice table); when None every population is scaled by 1/q.
    """
    nx, ny, nz = shape
    rng = np.random.Generator(np.random.PCG64(seed))
    w = np.full(q, 1.0 / q) if weights is None else np.asarray(weights, dtype=np.float64)
    noise = rng.standard_normal((q, nz, ny, nx))
    return w[:, None, None, None] * (1.0 + amp * noise)


def ensemble_viscosities(nbox: int, seed: int = 0, lo: float = 5e-5, hi: float = 5e-4) -> np.ndarray:
    """Per-box viscosities uniform in [lo, hi] from a seeded PCG64 generator."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return lo + (hi - lo) * rng.random(nbox)
