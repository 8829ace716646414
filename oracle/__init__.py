"""FP64 CPU oracle for the kinetic-closure lattice-Boltzmann update.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` load it; the product path never does.  It shares
no code with the CUDA library.  ``build()`` compiles ``lbm_oracle.c`` with gcc
(``-O2 -ffp-contract=off``, OpenMP) into ``oracle/liblbm_oracle.so``.

The algorithm is App. F of Marson & Malaspinas (arXiv 2605.19796): steps 1-7
of App. F.1, the KC-RB / KC-MP / KC-RR operational rules of App. F.2-F.4,
the product equilibrium Eq. (discrete_equilibrium), the finite-difference
strain Eqs. (fd), (strain_rate_discrete), (fd_boundary_lower/upper) and the
clipped turbulent rate Eq. (omega_sgs_operational).  The pins that tie it to
the paper and to mathematics live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")

BGK, KCMP, KCRB_HERMITE, KCRB_RAW, KCRR = 0, 1, 2, 3, 4
THETA = 1.0 / 3.0

_lib: Optional[ctypes.CDLL] = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain C, FP64, no FMA contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P = ctypes.POINTER
    dp, ip = P(ctypes.c_double), P(ctypes.c_int)
    c_int, c_double = ctypes.c_int, ctypes.c_double
    lib.orc_lattice_tables.argtypes = [c_int, ip, dp, ip]
    lib.orc_equilibrium.argtypes = [c_int, c_double, dp, dp]
    lib.orc_omega_sgs.argtypes = [c_double, c_double, c_double, c_double, c_double]
    lib.orc_omega_sgs.restype = c_double
    lib.orc_collide_cell.argtypes = [c_int, c_int, dp, dp, dp, c_double, c_double, c_double, dp, dp]
    lib.orc_closure_parts.argtypes = [c_int, c_int, dp, dp, c_double, c_double, c_double, dp, dp]
    lib.orc_strain_field.argtypes = [c_int, c_int, c_int, ip, dp, dp]
    lib.orc_run.argtypes = [c_int, c_int, c_int, c_int, c_int, ip, c_double, c_double, c_double, dp, dp, c_int]
    lib.orc_step_cell.argtypes = [c_int, c_int, c_double, c_double, c_double, dp, dp]
    lib.orc_init_equilibrium.argtypes = [c_int, c_int, c_int, c_int, dp, dp, dp]
    lib.orc_fields.argtypes = [c_int, c_int, c_int, c_int, dp, dp, dp, dp]
    lib.orc_diagnostics.argtypes = [c_int, c_int, c_int, c_int, ip, dp, dp, dp]
    lib.orc_dissipation.argtypes = [c_int, c_int, c_int, c_int, c_int, ip, c_double, c_double, c_double, dp, dp, dp]
    lib.orc_dissipation_pre.argtypes = [c_int, c_int, c_int, c_int, c_int, ip, c_double, c_double, c_double, dp, dp, dp]
    lib.orc_num_threads.restype = c_int
    lib.orc_set_num_threads.argtypes = [c_int]
    _lib = lib
    return lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def lattice(q: int):
    """Velocities c[q,3] (int), weights w[q], opposite index opp[q] in canonical order."""
    lib = _load()
    c = np.zeros(q * 3, dtype=np.int32)
    w = np.zeros(q, dtype=np.float64)
    opp = np.zeros(q, dtype=np.int32)
    _check(lib.orc_lattice_tables(q, _ip(c), _dp(w), _ip(opp)), "lattice")
    return c.reshape(q, 3), w, opp


def equilibrium(q: int, rho: float, u: Sequence[float]) -> np.ndarray:
    lib = _load()
    uu = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(q, dtype=np.float64)
    _check(lib.orc_equilibrium(q, float(rho), _dp(uu), _dp(out)), "equilibrium")
    return out


def omega_hat(nu: float) -> float:
    """Shifted molecular rate, Eq. (omega_t_discrete): (nu/theta + 1/2)^-1."""
    return 1.0 / (nu / THETA + 0.5)


def omega_sgs(tr_msgs: float, nu: float, c_nu: float, delta: float = 1.0) -> float:
    lib = _load()
    return lib.orc_omega_sgs(float(tr_msgs), float(nu), omega_hat(nu), float(c_nu), float(delta))


def collide_cell(q: int, closure: int, f: np.ndarray, S: np.ndarray, nu: float, c_nu: float,
                 delta: float = 1.0, F: Sequence[float] = (0.0, 0.0, 0.0)):
    """Post-collision populations of one cell for given pre-collision f and strain S (3x3)."""
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.float64)
    S9 = np.ascontiguousarray(np.asarray(S, dtype=np.float64).reshape(9))
    FF = np.ascontiguousarray(F, dtype=np.float64)
    out = np.zeros(q, dtype=np.float64)
    om = np.zeros(1, dtype=np.float64)
    _check(lib.orc_collide_cell(q, closure, _dp(f), _dp(S9), _dp(FF), float(nu), float(c_nu), float(delta),
                                _dp(out), _dp(om)), "collide_cell")
    return out, float(om[0])


def closure_parts(q: int, closure: int, f: np.ndarray, S: np.ndarray, nu: float, c_nu: float,
                  delta: float = 1.0):
    """(f0, f1, f_sgs, omega_s) of one cell: the equilibrium, the CE part and the
    SGS carrier the closure relaxes (App. F.2-F.4)."""
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.float64)
    S9 = np.ascontiguousarray(np.asarray(S, dtype=np.float64).reshape(9))
    parts = np.zeros(3 * q, dtype=np.float64)
    om = np.zeros(1, dtype=np.float64)
    _check(lib.orc_closure_parts(q, closure, _dp(f), _dp(S9), float(nu), float(c_nu), float(delta),
                                 _dp(parts), _dp(om)), "closure_parts")
    return parts[:q].copy(), parts[q:2 * q].copy(), parts[2 * q:].copy(), float(om[0])


def strain_field(u: np.ndarray, bc=(0, 0, 0)) -> np.ndarray:
    """S[3,3,nz,ny,nx] of a velocity field u[3,nz,ny,nx] (App. F.1 step 3)."""
    lib = _load()
    _, nz, ny, nx = u.shape
    uu = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros((9, nz, ny, nx), dtype=np.float64)
    b = np.ascontiguousarray(bc, dtype=np.int32)
    _check(lib.orc_strain_field(nx, ny, nz, _ip(b), _dp(uu), _dp(out)), "strain_field")
    return out.reshape(3, 3, nz, ny, nx)


def run(f: np.ndarray, nsteps: int, *, closure: int, nu: float, c_nu: float = 0.0, delta: float = 1.0,
        bc=(0, 0, 0), F: Sequence[float] = (0.0, 0.0, 0.0)) -> np.ndarray:
    """Advance populations f[q,nz,ny,nx] (post-collision state) by nsteps; returns a new array."""
    lib = _load()
    q, nz, ny, nx = f.shape
    out = np.array(f, dtype=np.float64, order="C", copy=True)
    b = np.ascontiguousarray(bc, dtype=np.int32)
    FF = np.ascontiguousarray(F, dtype=np.float64)
    _check(lib.orc_run(q, nx, ny, nz, closure, _ip(b), float(nu), float(c_nu), float(delta), _dp(FF),
                       _dp(out), int(nsteps)), "run")
    return out


def step_cell(block: np.ndarray, *, closure: int, nu: float, c_nu: float, delta: float = 1.0) -> np.ndarray:
    """Post-collision populations of the centre cell of a periodic 5x5x5 block [q,5,5,5] after one step."""
    lib = _load()
    q = block.shape[0]
    assert block.shape[1:] == (5, 5, 5)
    blk = np.ascontiguousarray(block, dtype=np.float64)
    out = np.zeros(q, dtype=np.float64)
    _check(lib.orc_step_cell(q, closure, float(nu), float(c_nu), float(delta), _dp(blk), _dp(out)), "step_cell")
    return out


def init_equilibrium(q: int, rho: Optional[np.ndarray], u: np.ndarray) -> np.ndarray:
    """f[q,nz,ny,nx] = f0(rho, u) at every node; rho None means 1."""
    lib = _load()
    _, nz, ny, nx = u.shape
    uu = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros((q, nz, ny, nx), dtype=np.float64)
    if rho is None:
        rp = ctypes.POINTER(ctypes.c_double)()
    else:
        rr = np.ascontiguousarray(rho, dtype=np.float64)
        rp = _dp(rr)
    _check(lib.orc_init_equilibrium(q, nx, ny, nz, rp, _dp(uu), _dp(out)), "init_equilibrium")
    return out


def fields(f: np.ndarray, F: Sequence[float] = (0.0, 0.0, 0.0)):
    """rho[nz,ny,nx], u[3,nz,ny,nx] of a stored (post-collision) population array
    (App. F.1 step 1); with a body force the reported velocity is (sum f c - F/2)/rho."""
    lib = _load()
    q, nz, ny, nx = f.shape
    ff = np.ascontiguousarray(f, dtype=np.float64)
    rho = np.zeros((nz, ny, nx), dtype=np.float64)
    u = np.zeros((3, nz, ny, nx), dtype=np.float64)
    FF = np.ascontiguousarray(F, dtype=np.float64)
    _check(lib.orc_fields(q, nx, ny, nz, _dp(FF), _dp(ff), _dp(rho), _dp(u)), "fields")
    return rho, u


def diagnostics(f: np.ndarray, bc=(0, 0, 0), F: Sequence[float] = (0.0, 0.0, 0.0)) -> np.ndarray:
    """[mass, momx, momy, momz, E_k, enstrophy, n_nonfinite, 0] (Sec. 7.1 averages)."""
    lib = _load()
    q, nz, ny, nx = f.shape
    ff = np.ascontiguousarray(f, dtype=np.float64)
    b = np.ascontiguousarray(bc, dtype=np.int32)
    FF = np.ascontiguousarray(F, dtype=np.float64)
    out = np.zeros(8, dtype=np.float64)
    _check(lib.orc_diagnostics(q, nx, ny, nz, _ip(b), _dp(FF), _dp(ff), _dp(out)), "diagnostics")
    return out


def _dissipation(fn, what, f, closure, nu, c_nu, delta, bc, F):
    lib = _load()
    q, nz, ny, nx = f.shape
    ff = np.ascontiguousarray(f, dtype=np.float64)
    b = np.ascontiguousarray(bc, dtype=np.int32)
    FF = np.ascontiguousarray(F, dtype=np.float64)
    out = np.zeros(2, dtype=np.float64)
    _check(getattr(lib, fn)(q, nx, ny, nz, closure, _ip(b), float(nu), float(c_nu), float(delta), _dp(FF), _dp(ff),
                            _dp(out)), what)
    return out


def dissipation(f: np.ndarray, *, closure: int, nu: float, c_nu: float = 0.0, delta: float = 1.0, bc=(0, 0, 0),
                F: Sequence[float] = (0.0, 0.0, 0.0)) -> np.ndarray:
    """[<2 rho nu_eff S:S>, <2 rho nu S:S>] of the state the next step collides:
    the stored post-collision populations f[q,nz,ny,nx] pull-streamed; nu_eff =
    theta (1/omega_s - 1/2) from the closure's clipped rate at each node."""
    return _dissipation("orc_dissipation", "dissipation", f, closure, nu, c_nu, delta, bc, F)


def dissipation_pre(f_pre: np.ndarray, *, closure: int, nu: float, c_nu: float = 0.0, delta: float = 1.0,
                    bc=(0, 0, 0), F: Sequence[float] = (0.0, 0.0, 0.0)) -> np.ndarray:
    """As dissipation() for a given pre-collision (already streamed) state."""
    return _dissipation("orc_dissipation_pre", "dissipation_pre", f_pre, closure, nu, c_nu, delta, bc, F)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(n: int) -> None:
    _load().orc_set_num_threads(int(n))
