"""Pins of the oracle's energy spectrum E(k) (oracle/spectrum.py) against what
the definition fixes: a single Fourier mode puts exactly A^2/4 in the shell of
its wave number (an axis mode and an oblique one, |k| = 5 from k = (3, 4) and
|k| = sqrt(3) rounding to shell 2), the shells sum to <|u|^2>/2 (Parseval), and
a planted mistake in the oracle's source (normalisation, the factor 1/2,
floor binning, the max-norm instead of |k|) fails one of these.  The package's
torch spectrum (used by the learned-closure and precision studies) is checked
against the oracle on a random field."""
import math
import os

import numpy as np
import pytest

import oracle.spectrum as osp

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "spectrum.py")


def _grid(n):
    x = np.arange(n, dtype=np.float64)
    return np.meshgrid(x, x, x, indexing="ij")  # z, y, x


def _pins(spectrum, all_shells):
    """Raises AssertionError unless the pins hold for these functions."""
    n, A = 16, 0.3
    z, y, x = _grid(n)
    # axis mode along z in u_x: A sin(2 pi k0 z / N)
    for k0 in (1, 3, 7):
        u = np.zeros((3, n, n, n))
        u[0] = A * np.sin(2 * math.pi * k0 * z / n)
        e = spectrum(u)
        assert e.shape == (n // 2,)
        assert abs(e[k0] - A * A / 4) <= 1e-14, (k0, e[k0])
        assert np.abs(np.delete(e, k0)).max() <= 1e-14
    # oblique mode in u_y: A cos(2 pi (3 x + 4 y) / N), |k| = 5
    u = np.zeros((3, n, n, n))
    u[1] = A * np.cos(2 * math.pi * (3 * x + 4 * y) / n)
    e = spectrum(u)
    assert abs(e[5] - A * A / 4) <= 1e-14 and np.abs(np.delete(e, 5)).max() <= 1e-14
    # |k| = sqrt(3) = 1.73 belongs to shell 2 (k - 1/2 <= |k| < k + 1/2)
    u = np.zeros((3, n, n, n))
    u[2] = A * np.sin(2 * math.pi * (x + y + z) / n)
    e = spectrum(u)
    assert abs(e[2] - A * A / 4) <= 1e-14 and abs(e[1]) <= 1e-14
    # Parseval on a random field
    rng = np.random.default_rng(5)
    u = rng.standard_normal((3, n, n, n))
    es = all_shells(u)
    assert abs(es.sum() - 0.5 * (u ** 2).sum(axis=0).mean()) <= 1e-12 * es.sum()
    assert np.allclose(spectrum(u), es[: n // 2], rtol=0, atol=1e-15)


def test_spectrum_pins():
    _pins(osp.spectrum, osp.all_shells)


MUTATIONS = [
    ("/ float(n) ** 3", "/ float(n) ** 1.5"),           # normalisation
    ("e = 0.5 * (uh.real", "e = 1.0 * (uh.real"),       # the factor 1/2 (both functions)
    ("np.floor(kmag + 0.5)", "np.floor(kmag)"),         # floor binning
    ("np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)\n    shell", "np.maximum(np.maximum(np.abs(kx), np.abs(ky)), np.abs(kz))\n    shell"),
]


@pytest.mark.parametrize("old,new", MUTATIONS)
def test_planted_mistakes_fail_the_pins(old, new):
    src = open(SRC).read()
    assert old in src, old
    ns = {}
    exec(compile(src.replace(old, new), "mutated_spectrum", "exec"), ns)
    with pytest.raises(AssertionError):
        _pins(ns["spectrum"], ns["all_shells"])


def test_package_spectrum_equals_oracle():
    torch = pytest.importorskip("torch")
    from paper_2605_19796_gb300 import learned

    rng = np.random.default_rng(11)
    u = rng.standard_normal((3, 24, 24, 24))
    ep = learned.spectrum(torch.from_numpy(u)).numpy()
    eo = osp.spectrum(u)
    assert ep.shape == eo.shape
    assert np.abs(ep - eo).max() <= 1e-12 * eo.max()
