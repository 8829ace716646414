"""Thin ctypes binding of the C ABI in ``include/lbm.h`` (liblbm.so).

Argument marshalling only: every step of the lattice update runs in the
library's CUDA kernels.  Importing this module loads ``csrc/liblbm.so`` and
raises ``ImportError`` when it has not been built (``build.build()``); there is
no CPU fallback.

The functions keep the C names (``lbm_create``, ``lbm_step`` ...); ``Solver``
wraps a handle with numpy/torch-friendly methods.
"""
from __future__ import annotations

import ctypes
import os
import weakref
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "csrc", "liblbm.so")

LBM_OK = 0
LBM_ERR_ARG, LBM_ERR_OOM, LBM_ERR_CUDA, LBM_ERR_NONFINITE = -1, -2, -3, -4
LBM_ERR_TIMEOUT, LBM_ERR_UNSUPPORTED, LBM_ERR_IO = -5, -6, -7
LBM_D3Q19, LBM_D3Q27 = 19, 27
LBM_BGK, LBM_KCMP, LBM_KCRB_HERMITE, LBM_KCRB_RAW, LBM_KCRR, LBM_LEARNED = 0, 1, 2, 3, 4, 5
LBM_FP64, LBM_FP32, LBM_FP16_SHIFTED, LBM_BF16_SHIFTED = 0, 1, 2, 3
LBM_PERIODIC, LBM_BOUNCEBACK = 0, 1

CLOSURES = {"bgk": LBM_BGK, "kcmp": LBM_KCMP, "kcrb_hermite": LBM_KCRB_HERMITE, "kcrb_raw": LBM_KCRB_RAW,
            "kcrr": LBM_KCRR, "learned": LBM_LEARNED}
STORAGES = {"fp64": LBM_FP64, "fp32": LBM_FP32, "fp16": LBM_FP16_SHIFTED, "bf16": LBM_BF16_SHIFTED}
# closure coefficients used by the paper (Sec. 7): KC-MP 0.035, KC-RB and KC-RR 0.02
DEFAULT_CNU = {LBM_BGK: 0.0, LBM_KCMP: 0.035, LBM_KCRB_HERMITE: 0.02, LBM_KCRB_RAW: 0.02, LBM_KCRR: 0.02,
               LBM_LEARNED: 0.035}
EXPORTS = ["lbm_config_default", "lbm_create", "lbm_destroy", "lbm_init_velocity", "lbm_init_velocity_device",
           "lbm_step", "lbm_moments", "lbm_moments_device", "lbm_diagnostics", "lbm_get_populations",
           "lbm_set_populations", "lbm_probe", "lbm_population_buffer", "lbm_synchronize", "lbm_save", "lbm_load",
           "lbm_step_count", "lbm_kernel_launches", "lbm_last_error", "lbm_abi_version",
           "lbm_diagnostics_noalloc", "lbm_autotune", "lbm_launch_config", "lbm_mlp_param_count",
           "lbm_mlp_workspace_floats", "lbm_mlp_forward", "lbm_mlp_grad", "lbm_mlp_adamw", "lbm_box_filter",
           "lbm_closure_features", "lbm_closure_strain", "lbm_set_learned_closure", "lbm_mlp_packed_bytes", "lbm_mlp_pack",
           "lbm_mlp_forward_tc", "lbm_wait_selftest", "lbm_host_alloc", "lbm_host_free",
           "lbm_init_velocity_f32", "lbm_moments_f32", "lbm_read_learned_closure",
           "lbm_set_learned_closure_file"]


class lbm_config(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("nbatch", ctypes.c_int), ("nu", ctypes.POINTER(ctypes.c_double)), ("closure", ctypes.c_int),
                ("c_nu", ctypes.c_double), ("delta", ctypes.c_double), ("storage", ctypes.c_int),
                ("bc", ctypes.c_int * 3), ("force", ctypes.c_double * 3), ("cuda_stream", ctypes.c_void_p),
                ("tile_y", ctypes.c_int), ("zchunk", ctypes.c_int), ("variant", ctypes.c_int),
                ("disable_graphs", ctypes.c_int)]


class LbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"liblbm error {code}: {msg}")
        self.code = code


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run paper_2605_19796_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    dp = P(ctypes.c_double)
    vp = ctypes.c_void_p
    H = vp
    lib.lbm_config_default.argtypes = [P(lbm_config)]
    lib.lbm_config_default.restype = None
    lib.lbm_create.argtypes = [P(lbm_config), P(vp)]
    lib.lbm_destroy.argtypes = [H]
    lib.lbm_destroy.restype = None
    lib.lbm_init_velocity.argtypes = [H, dp, dp]
    fp = P(ctypes.c_float)
    lib.lbm_read_learned_closure.argtypes = [ctypes.c_char_p, fp, ctypes.c_int, fp, ctypes.c_int]
    lib.lbm_set_learned_closure_file.argtypes = [H, ctypes.c_char_p]
    lib.lbm_init_velocity_f32.argtypes = [H, fp, fp]
    lib.lbm_moments_f32.argtypes = [H, fp, fp]
    lib.lbm_init_velocity_device.argtypes = [H, vp, vp]
    lib.lbm_step.argtypes = [H, ctypes.c_int]
    lib.lbm_moments.argtypes = [H, dp, dp]
    lib.lbm_moments_device.argtypes = [H, vp, vp]
    lib.lbm_diagnostics.argtypes = [H, ctypes.c_int, dp]
    lib.lbm_get_populations.argtypes = [H, dp]
    lib.lbm_set_populations.argtypes = [H, dp]
    lib.lbm_probe.argtypes = [H, ctypes.c_int, P(ctypes.c_int), ctypes.c_int, dp]
    lib.lbm_population_buffer.argtypes = [H, P(vp), P(ctypes.c_int)]
    lib.lbm_synchronize.argtypes = [H]
    lib.lbm_save.argtypes = [H, ctypes.c_char_p]
    lib.lbm_load.argtypes = [H, ctypes.c_char_p]
    lib.lbm_step_count.argtypes = [H]
    lib.lbm_step_count.restype = ctypes.c_int64
    lib.lbm_kernel_launches.argtypes = [H]
    lib.lbm_kernel_launches.restype = ctypes.c_int64
    lib.lbm_diagnostics_noalloc.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            P(ctypes.c_int), dp, vp, vp]
    fl = ctypes.c_float
    lib.lbm_mlp_param_count.restype = ctypes.c_int
    lib.lbm_mlp_workspace_floats.argtypes = [ctypes.c_int]
    lib.lbm_mlp_workspace_floats.restype = ctypes.c_longlong
    lib.lbm_mlp_forward.argtypes = [vp, vp, ctypes.c_int, vp, vp, vp]
    lib.lbm_mlp_grad.argtypes = [vp, vp, vp, ctypes.c_int, vp, vp, dp, vp]
    lib.lbm_mlp_adamw.argtypes = [vp, vp, vp, vp, ctypes.c_int, fl, fl, fl, fl, fl, vp]
    lib.lbm_box_filter.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_double, ctypes.c_int, vp, vp, vp]
    lib.lbm_closure_features.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, vp, vp, vp, vp, vp]
    lib.lbm_closure_strain.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp]
    lib.lbm_set_learned_closure.argtypes = [H, P(ctypes.c_float), P(ctypes.c_float)]
    lib.lbm_mlp_packed_bytes.restype = ctypes.c_longlong
    lib.lbm_mlp_pack.argtypes = [P(ctypes.c_float), P(ctypes.c_float), vp]
    lib.lbm_mlp_forward_tc.argtypes = [vp, vp, ctypes.c_int, vp, vp]
    lib.lbm_wait_selftest.argtypes = [H, ctypes.c_int]
    lib.lbm_host_alloc.argtypes = [ctypes.c_size_t, P(vp)]
    lib.lbm_host_free.argtypes = [vp]
    lib.lbm_autotune.argtypes = [H, ctypes.c_int]
    lib.lbm_launch_config.argtypes = [H, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int)]
    lib.lbm_last_error.restype = ctypes.c_char_p
    lib.lbm_abi_version.restype = ctypes.c_int
    return lib


LIB = _load()


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return ctypes.POINTER(ctypes.c_double)()
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "expected a C-contiguous float64 array"
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _fp(a: Optional[np.ndarray]):
    if a is None:
        return ctypes.POINTER(ctypes.c_float)()
    assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"], "expected a C-contiguous float32 array"
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _check(rc: int) -> None:
    if rc != LBM_OK:
        raise LbmError(rc, LIB.lbm_last_error().decode())


# ---------------------------------------------------------------- C names

def lbm_config_default() -> lbm_config:
    cfg = lbm_config()
    LIB.lbm_config_default(ctypes.byref(cfg))
    return cfg


def lbm_create(cfg: lbm_config) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(LIB.lbm_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def lbm_destroy(h) -> None:
    LIB.lbm_destroy(h)


def lbm_init_velocity(h, rho: Optional[np.ndarray], u: np.ndarray) -> None:
    _check(LIB.lbm_init_velocity(h, _dp(rho), _dp(u)))


def lbm_init_velocity_f32(h, rho: Optional[np.ndarray], u: np.ndarray) -> None:
    _check(LIB.lbm_init_velocity_f32(h, _fp(rho), _fp(u)))


def lbm_moments_f32(h, rho: Optional[np.ndarray], u: Optional[np.ndarray]) -> None:
    _check(LIB.lbm_moments_f32(h, _fp(rho), _fp(u)))


def lbm_init_velocity_device(h, rho_ptr: int, u_ptr: int) -> None:
    _check(LIB.lbm_init_velocity_device(h, ctypes.c_void_p(rho_ptr or None), ctypes.c_void_p(u_ptr)))


def lbm_step(h, nsteps: int) -> None:
    _check(LIB.lbm_step(h, int(nsteps)))


def lbm_moments(h, rho: Optional[np.ndarray], u: Optional[np.ndarray]) -> None:
    _check(LIB.lbm_moments(h, _dp(rho), _dp(u)))


def lbm_moments_device(h, rho_ptr: int, u_ptr: int) -> None:
    _check(LIB.lbm_moments_device(h, ctypes.c_void_p(rho_ptr or None), ctypes.c_void_p(u_ptr or None)))


def lbm_host_alloc(nbytes: int) -> int:
    p = ctypes.c_void_p()
    _check(LIB.lbm_host_alloc(ctypes.c_size_t(int(nbytes)), ctypes.byref(p)))
    return p.value


def lbm_host_free(ptr: int) -> None:
    _check(LIB.lbm_host_free(ctypes.c_void_p(ptr or None)))


def host_empty(shape, dtype=np.float64) -> np.ndarray:
    """A NumPy array in page-locked host memory from lbm_host_alloc (the fast
    path for the host-pointer transfers); the memory is released with
    lbm_host_free when the array and all its views are gone."""
    dt = np.dtype(dtype)
    n = int(np.prod(shape)) if len(tuple(shape)) else 1
    nbytes = max(1, n) * dt.itemsize
    ptr = lbm_host_alloc(nbytes)
    buf = (ctypes.c_char * nbytes).from_address(ptr)
    arr = np.frombuffer(buf, dtype=dt, count=n).reshape(shape)
    weakref.finalize(buf, lbm_host_free, ptr)
    return arr


DIAG_VALUES = 10  # LBM_DIAG_VALUES of include/lbm.h


def lbm_diagnostics(h, box: int, out: np.ndarray) -> None:
    """out: FP64 array of DIAG_VALUES values (layout in include/lbm.h)."""
    if out.dtype != np.float64 or out.size < DIAG_VALUES:
        raise ValueError("out must hold %d float64 values" % DIAG_VALUES)
    _check(LIB.lbm_diagnostics(h, int(box), _dp(out)))


def lbm_get_populations(h, f: np.ndarray) -> None:
    _check(LIB.lbm_get_populations(h, _dp(f)))


def lbm_set_populations(h, f: np.ndarray) -> None:
    _check(LIB.lbm_set_populations(h, _dp(f)))


def lbm_probe(h, box: int, xyz: np.ndarray, out: np.ndarray) -> None:
    xyz = np.ascontiguousarray(xyz, dtype=np.int32)
    _check(LIB.lbm_probe(h, int(box), xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), int(xyz.shape[0]), _dp(out)))


def lbm_population_buffer(h):
    p = ctypes.c_void_p()
    e = ctypes.c_int()
    _check(LIB.lbm_population_buffer(h, ctypes.byref(p), ctypes.byref(e)))
    return p.value, e.value


def lbm_synchronize(h) -> None:
    _check(LIB.lbm_synchronize(h))


def lbm_save(h, path: str) -> None:
    _check(LIB.lbm_save(h, path.encode()))


def lbm_load(h, path: str) -> None:
    _check(LIB.lbm_load(h, path.encode()))


def lbm_step_count(h) -> int:
    return int(LIB.lbm_step_count(h))


def lbm_kernel_launches(h) -> int:
    return int(LIB.lbm_kernel_launches(h))


def lbm_diagnostics_noalloc(f_ptr: int, lattice: int, storage: int, nx: int, ny: int, nz: int, bc=None,
                            force=None, out_ptr: int = 0, stream=None) -> None:
    """Allocation-free diagnostics of one box (see include/lbm.h): f_ptr and
    out_ptr are device addresses; enqueued on ``stream``."""
    b = None if bc is None else np.ascontiguousarray(bc, dtype=np.int32)
    F = None if force is None else np.ascontiguousarray(force, dtype=np.float64)
    sh = _stream_handle(stream)
    _check(LIB.lbm_diagnostics_noalloc(ctypes.c_void_p(f_ptr), int(lattice), int(storage), int(nx), int(ny), int(nz),
                                       None if b is None else b.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                       _dp(F), ctypes.c_void_p(out_ptr), ctypes.c_void_p(sh) if sh else None))


def lbm_autotune(h, trials: int = 3) -> None:
    _check(LIB.lbm_autotune(h, int(trials)))


def lbm_launch_config(h):
    v, t, z = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(LIB.lbm_launch_config(h, ctypes.byref(v), ctypes.byref(t), ctypes.byref(z)))
    return {"variant": v.value, "tile_y": t.value, "zchunk": z.value}


def _vp(ptr):
    return ctypes.c_void_p(int(ptr)) if ptr else None


def lbm_mlp_param_count() -> int:
    return int(LIB.lbm_mlp_param_count())


def lbm_mlp_workspace_floats(n: int) -> int:
    return int(LIB.lbm_mlp_workspace_floats(int(n)))


def lbm_mlp_forward(params, xs, n, ys, workspace, stream=None) -> None:
    """Device pointers (ints); see include/lbm.h."""
    _check(LIB.lbm_mlp_forward(_vp(params), _vp(xs), int(n), _vp(ys), _vp(workspace), _vp(_stream_handle(stream))))


def lbm_mlp_grad(params, xs, ts, n, grad, workspace, stream=None, want_loss=True):
    loss = ctypes.c_double(0.0)
    _check(LIB.lbm_mlp_grad(_vp(params), _vp(xs), _vp(ts), int(n), _vp(grad), _vp(workspace),
                            ctypes.byref(loss) if want_loss else None, _vp(_stream_handle(stream))))
    return loss.value if want_loss else None


def lbm_mlp_adamw(params, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0,
                  stream=None) -> None:
    _check(LIB.lbm_mlp_adamw(_vp(params), _vp(grad), _vp(m), _vp(v), int(step), float(lr), float(beta1),
                             float(beta2), float(eps), float(weight_decay), _vp(_stream_handle(stream))))


def lbm_box_filter(f_ptr, lattice, storage, nx, ny, nz, factor, fc_ptr, msgs_ptr, stream=None,
                   neq_scale: float = 1.0, pull: bool = False) -> None:
    _check(LIB.lbm_box_filter(_vp(f_ptr), int(lattice), int(storage), int(nx), int(ny), int(nz), int(factor),
                              float(neq_scale), int(bool(pull)), _vp(fc_ptr), _vp(msgs_ptr),
                              _vp(_stream_handle(stream))))


def lbm_closure_features(f_ptr, lattice, nx, ny, nz, nu, msgs_ptr, x_ptr, t_ptr, kcmp_ptr=0, stream=None) -> None:
    _check(LIB.lbm_closure_features(_vp(f_ptr), int(lattice), int(nx), int(ny), int(nz), float(nu), _vp(msgs_ptr),
                                    _vp(x_ptr), _vp(t_ptr), _vp(kcmp_ptr), _vp(_stream_handle(stream))))


def lbm_closure_strain(f_ptr, lattice, nx, ny, nz, s_ptr, stream=None) -> None:
    _check(LIB.lbm_closure_strain(_vp(f_ptr), int(lattice), int(nx), int(ny), int(nz), _vp(s_ptr),
                                  _vp(_stream_handle(stream))))


def lbm_mlp_pack(params: np.ndarray, stats: np.ndarray) -> np.ndarray:
    """Packed network block (bytes) of the fused inference."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    st = np.ascontiguousarray(stats, dtype=np.float32)
    out = np.zeros(int(LIB.lbm_mlp_packed_bytes()), dtype=np.uint8)
    fp = ctypes.POINTER(ctypes.c_float)
    _check(LIB.lbm_mlp_pack(p.ctypes.data_as(fp), st.ctypes.data_as(fp), out.ctypes.data_as(ctypes.c_void_p)))
    return out


def lbm_mlp_forward_tc(packed_ptr, x_ptr, n, y_ptr, stream=None) -> None:
    _check(LIB.lbm_mlp_forward_tc(_vp(packed_ptr), _vp(x_ptr), int(n), _vp(y_ptr), _vp(_stream_handle(stream))))


def lbm_wait_selftest(h, polls: int) -> int:
    """Return code of the bounded-wait self-test (LBM_ERR_TIMEOUT when the error path works)."""
    return int(LIB.lbm_wait_selftest(h, int(polls)))


def write_learned_closure(path: str, params: np.ndarray, stats: np.ndarray) -> None:
    """The network file lbm_read_learned_closure reads: b"LBMMLP01", int32
    counts (9414, 32), FP32 parameters, FP32 statistics, little-endian."""
    p = np.ascontiguousarray(params, dtype="<f4").ravel()
    st = np.ascontiguousarray(stats, dtype="<f4").ravel()
    assert p.size == lbm_mlp_param_count() and st.size == 32
    with open(path, "wb") as fp:
        fp.write(b"LBMMLP01")
        fp.write(np.array([p.size, st.size], dtype="<i4").tobytes())
        fp.write(p.tobytes())
        fp.write(st.tobytes())


def lbm_read_learned_closure(path: str):
    """(params [9414], stats [32]) float32 from a network file."""
    p = np.empty(lbm_mlp_param_count(), dtype=np.float32)
    st = np.empty(32, dtype=np.float32)
    _check(LIB.lbm_read_learned_closure(os.fsencode(path), _fp(p), p.size, _fp(st), st.size))
    return p, st


def lbm_set_learned_closure_file(h, path: str) -> None:
    _check(LIB.lbm_set_learned_closure_file(h, os.fsencode(path)))


def lbm_set_learned_closure(h, params: np.ndarray, stats: np.ndarray) -> None:
    p = np.ascontiguousarray(params, dtype=np.float32)
    st = np.ascontiguousarray(stats, dtype=np.float32)
    assert p.size == lbm_mlp_param_count() and st.size == 32
    fp = ctypes.POINTER(ctypes.c_float)
    _check(LIB.lbm_set_learned_closure(h, p.ctypes.data_as(fp), st.ctypes.data_as(fp)))


def lbm_last_error() -> str:
    return LIB.lbm_last_error().decode()


def lbm_abi_version() -> int:
    return int(LIB.lbm_abi_version())


# ---------------------------------------------------------------- wrapper

def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


class Solver:
    """One handle: ``Solver(27, (nx, ny, nz), nu=1e-4, closure="kcmp", storage="fp32")``.

    Fields use the layouts of the C ABI: rho[nbatch, nz, ny, nx],
    u[3, nbatch, nz, ny, nx] (squeezed to [nz, ny, nx] / [3, nz, ny, nx] for
    one box), populations [nbatch, q, nz, ny, nx].
    """

    def __init__(self, lattice: int, shape: Sequence[int], nu, *, closure="kcmp", c_nu: Optional[float] = None,
                 delta: float = 1.0, storage="fp32", bc=(0, 0, 0), force=(0.0, 0.0, 0.0), stream=None,
                 nbatch: int = 1, tile_y: int = 0, zchunk: int = 0, variant: int = 0,
                 disable_graphs: bool = False):
        cfg = lbm_config_default()
        cfg.lattice = int(lattice)
        cfg.nx, cfg.ny, cfg.nz = (int(v) for v in shape)
        cfg.nbatch = int(nbatch)
        self._nu = np.ascontiguousarray(np.broadcast_to(np.asarray(nu, dtype=np.float64), (nbatch,)))
        cfg.nu = _dp(self._nu)
        cfg.closure = CLOSURES[closure] if isinstance(closure, str) else int(closure)
        cfg.c_nu = DEFAULT_CNU[cfg.closure] if c_nu is None else float(c_nu)
        cfg.delta = float(delta)
        cfg.storage = STORAGES[storage] if isinstance(storage, str) else int(storage)
        for k in range(3):
            cfg.bc[k] = int(bc[k])
            cfg.force[k] = float(force[k])
        sh = _stream_handle(stream)
        cfg.cuda_stream = ctypes.c_void_p(sh) if sh else None
        cfg.tile_y = int(tile_y)
        cfg.zchunk = int(zchunk)
        cfg.variant = int(variant)
        cfg.disable_graphs = int(bool(disable_graphs))
        self.cfg = cfg
        self.q = cfg.lattice
        self.shape = (cfg.nx, cfg.ny, cfg.nz)
        self.nbatch = cfg.nbatch
        self.h = lbm_create(cfg)

    # -- lifetime
    def close(self) -> None:
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- state
    @property
    def ncell(self) -> int:
        nx, ny, nz = self.shape
        return nx * ny * nz

    def _fshape(self):
        nx, ny, nz = self.shape
        return (self.nbatch, nz, ny, nx)

    def init_velocity(self, rho: Optional[np.ndarray], u: np.ndarray) -> None:
        """float32 u goes through lbm_init_velocity_f32 (rho converted to float32),
        anything else through lbm_init_velocity as float64."""
        dt = np.float32 if np.asarray(u).dtype == np.float32 else np.float64
        u = np.ascontiguousarray(u, dtype=dt).reshape(3, -1)
        r = None if rho is None else np.ascontiguousarray(rho, dtype=dt).reshape(-1)
        (lbm_init_velocity_f32 if dt == np.float32 else lbm_init_velocity)(self.h, r, u)

    def init_velocity_device(self, rho, u) -> None:
        """rho, u: CUDA float64 tensors (rho may be None) in the C ABI layouts."""
        lbm_init_velocity_device(self.h, 0 if rho is None else rho.data_ptr(), u.data_ptr())

    def step(self, n: int = 1) -> None:
        lbm_step(self.h, n)

    def moments(self, dtype=np.float64):
        """rho, u as float64 (lbm_moments) or float32 (lbm_moments_f32)."""
        dt = np.dtype(dtype)
        assert dt in (np.float64, np.float32), "moments come as float64 or float32"
        rho = np.empty(self._fshape(), dtype=dt)
        u = np.empty((3,) + self._fshape(), dtype=dt)
        (lbm_moments_f32 if dt == np.float32 else lbm_moments)(self.h, rho, u)
        if self.nbatch == 1:
            return rho[0], u[:, 0]
        return rho, u

    def moments_device(self, rho, u) -> None:
        lbm_moments_device(self.h, 0 if rho is None else rho.data_ptr(), 0 if u is None else u.data_ptr())

    def diagnostics(self, box: int = 0) -> np.ndarray:
        """[mass, momentum x3, E_k, enstrophy, non-finite cells, max|u|,
        <2 rho nu_eff S:S>, <2 rho nu S:S>] (include/lbm.h, lbm_diagnostics)."""
        out = np.zeros(DIAG_VALUES, dtype=np.float64)
        lbm_diagnostics(self.h, box, out)
        return out

    def get_populations(self) -> np.ndarray:
        nb, nz, ny, nx = self._fshape()
        f = np.empty((nb, self.q, nz, ny, nx), dtype=np.float64)
        lbm_get_populations(self.h, f)
        return f[0] if nb == 1 else f

    def set_populations(self, f: np.ndarray) -> None:
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.size == self.nbatch * self.q * self.ncell
        lbm_set_populations(self.h, f)

    def probe(self, xyz, box: int = 0) -> np.ndarray:
        """FP64 populations [n, q] of the cells xyz[n, 3] = (x, y, z) (wrapped periodically)."""
        xyz = np.ascontiguousarray(np.asarray(xyz).reshape(-1, 3), dtype=np.int32)
        out = np.empty((xyz.shape[0], self.q), dtype=np.float64)
        lbm_probe(self.h, box, xyz, out)
        return out

    def population_buffer(self):
        return lbm_population_buffer(self.h)

    def synchronize(self) -> None:
        lbm_synchronize(self.h)

    def save(self, path: str) -> None:
        lbm_save(self.h, path)

    def load(self, path: str) -> None:
        lbm_load(self.h, path)

    def set_learned_closure(self, params: np.ndarray, stats: np.ndarray) -> None:
        lbm_set_learned_closure(self.h, params, stats)

    def set_learned_closure_file(self, path: str) -> None:
        lbm_set_learned_closure_file(self.h, path)

    def autotune(self, trials: int = 3) -> dict:
        lbm_autotune(self.h, trials)
        return lbm_launch_config(self.h)

    @property
    def launch_config(self) -> dict:
        return lbm_launch_config(self.h)

    @property
    def step_count(self) -> int:
        return lbm_step_count(self.h)

    @property
    def kernel_launches(self) -> int:
        return lbm_kernel_launches(self.h)
