"""FP64 energy spectrum of a periodic velocity field (test infrastructure only).

The paper compares turbulent kinetic energy spectra E(k) of the Taylor-Green
runs (Sec. 7.1, the TKE spectra figures) without stating the binning or the
normalisation.  Reading used here: the discrete Fourier coefficients
normalised by the number of nodes,

    u_hat(k) = (1/N^3) sum_x u(x) exp(-2 pi i k.x / N),

and shells of unit width centred on the integers,

    E(k) = 1/2 sum_{k' : k - 1/2 <= |k'| < k + 1/2} |u_hat(k')|^2,

with |k'| the Euclidean norm of the integer wave vector (components in
-N/2 .. N/2 - 1).  With this normalisation sum_k E(k) = <|u|^2> / 2 (Parseval),
and a single mode A sin(2 pi k0 z / N) e_x puts A^2/4 in shell k0.  Shells up
to N/2 - 1 are returned (those fully inside the resolved cube); the corners of
the cube (|k'| >= N/2) are left out.  Plain numpy, written for checking by eye.
"""
from __future__ import annotations

import numpy as np


def spectrum(u: np.ndarray) -> np.ndarray:
    """E(k), k = 0 .. N/2 - 1, of u[3][N][N][N] (periodic cube, any float dtype)."""
    u = np.asarray(u, dtype=np.float64)
    assert u.ndim == 4 and u.shape[0] == 3 and u.shape[1] == u.shape[2] == u.shape[3], u.shape
    n = u.shape[-1]
    uh = np.fft.fftn(u, axes=(1, 2, 3)) / float(n) ** 3
    e = 0.5 * (uh.real ** 2 + uh.imag ** 2).sum(axis=0)
    k1 = np.fft.fftfreq(n, d=1.0 / n)  # integer wave numbers, -N/2 .. N/2 - 1
    kz, ky, kx = np.meshgrid(k1, k1, k1, indexing="ij")
    kmag = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    shell = np.floor(kmag + 0.5).astype(np.int64)  # k - 1/2 <= |k'| < k + 1/2
    out = np.zeros(n // 2, dtype=np.float64)
    inside = shell < n // 2
    np.add.at(out, shell[inside], e[inside])
    return out


def all_shells(u: np.ndarray) -> np.ndarray:
    """E(k) over every shell, the cube's corners included (sums to <|u|^2>/2)."""
    u = np.asarray(u, dtype=np.float64)
    n = u.shape[-1]
    uh = np.fft.fftn(u, axes=(1, 2, 3)) / float(n) ** 3
    e = 0.5 * (uh.real ** 2 + uh.imag ** 2).sum(axis=0)
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    kz, ky, kx = np.meshgrid(k1, k1, k1, indexing="ij")
    shell = np.floor(np.sqrt(kx ** 2 + ky ** 2 + kz ** 2) + 0.5).astype(np.int64)
    out = np.zeros(int(shell.max()) + 1, dtype=np.float64)
    np.add.at(out, shell.ravel(), e.ravel())
    return out
