"""CPU-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every entry point include/lbm.h declares, the binding wraps exactly
those, and configuration errors are rejected before any device work."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lbm():
    from paper_2605_19796_gb300 import build

    build.build()
    from paper_2605_19796_gb300 import lbm as _lbm

    return _lbm


def _declared():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src)))


def test_header_symbols_exported(lbm):
    names = _declared()
    assert len(names) >= 20
    lib = ctypes.CDLL(lbm.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(lbm.EXPORTS) == names


def test_abi_version(lbm):
    assert lbm.lbm_abi_version() == 2


def test_config_default(lbm):
    cfg = lbm.lbm_config_default()
    assert (cfg.lattice, cfg.nx, cfg.nbatch, cfg.closure, cfg.storage) == (27, 32, 1, lbm.LBM_KCMP, lbm.LBM_FP32)
    assert cfg.c_nu == 0.035 and cfg.delta == 1.0


def _cfg(lbm, **kw):
    cfg = lbm.lbm_config_default()
    nu = np.array([1e-4])
    cfg.nu = nu.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    for k, v in kw.items():
        if k == "bc":
            for a in range(3):
                cfg.bc[a] = v[a]
        elif k == "force":
            for a in range(3):
                cfg.force[a] = v[a]
        else:
            setattr(cfg, k, v)
    return cfg, nu


@pytest.mark.parametrize("kw,code", [
    (dict(lattice=20), -1), (dict(nx=0), -1), (dict(nbatch=0), -1), (dict(closure=9), -1),
    (dict(storage=7), -1), (dict(c_nu=-1.0), -1), (dict(delta=0.0), -1),
    (dict(lattice=19, closure=4), -6), (dict(bc=(1, 0, 0)), -6), (dict(bc=(0, 0, 1)), -6),
    (dict(force=(1e-5, 0.0, 0.0)), -6), (dict(bc=(0, 1, 0), ny=2), -1), (dict(tile_y=5), -6),
    (dict(nx=2048, ny=2048, nz=1024), -1),
    # retired and unknown kernel variants; variants not built for the storage or box
    (dict(variant=2), -1), (dict(variant=6), -1), (dict(variant=11), -1),     (dict(variant=15), -6), (dict(variant=15, closure=5, storage=0), -6), (dict(variant=15, closure=5, tile_y=8), -6),
    (dict(variant=16, nx=64), -6), (dict(variant=16, nx=64, tile_y=16, closure=5), -6),
    (dict(variant=16, storage=0, nx=128), -6), (dict(variant=17), -1),
    (dict(variant=14, nx=44), -6), (dict(variant=14, storage=0), -6),
    (dict(variant=14, closure=4, bc=(0, 1, 0), ny=32), -6), (dict(variant=16, closure=2, bc=(0, 1, 0), ny=32, nx=128), -6),
    (dict(variant=13, storage=2), -6),
    (dict(variant=9), -1), (dict(variant=4), -1),
])
def test_bad_config_rejected_before_device_work(lbm, kw, code):
    cfg, nu = _cfg(lbm, **kw)
    h = ctypes.c_void_p()
    rc = lbm.LIB.lbm_create(ctypes.byref(cfg), ctypes.byref(h))
    assert rc == code, lbm.lbm_last_error()
    assert h.value is None
    assert lbm.lbm_last_error() != ""


def test_null_arguments(lbm):
    assert lbm.LIB.lbm_create(None, None) == lbm.LBM_ERR_ARG
    assert lbm.LIB.lbm_step(None, 1) == lbm.LBM_ERR_ARG
    assert lbm.LIB.lbm_step_count(None) == -1
    assert lbm.LIB.lbm_init_velocity_f32(None, None, None) == lbm.LBM_ERR_ARG
    assert lbm.LIB.lbm_moments_f32(None, None, None) == lbm.LBM_ERR_ARG
    lbm.LIB.lbm_destroy(None)


def test_host_alloc_argument_checks_need_no_device(lbm):
    """lbm_host_alloc refuses a zero size or a NULL output before any CUDA call;
    lbm_host_free ignores NULL."""
    p = ctypes.c_void_p()
    assert lbm.LIB.lbm_host_alloc(ctypes.c_size_t(0), ctypes.byref(p)) == lbm.LBM_ERR_ARG
    assert p.value is None
    assert lbm.LIB.lbm_host_alloc(ctypes.c_size_t(64), None) == lbm.LBM_ERR_ARG
    assert lbm.LIB.lbm_host_free(None) == lbm.LBM_OK


def test_learned_closure_file_round_trip_and_errors(lbm, tmp_path):
    """The network file (magic, int32 counts, FP32 parameters and statistics)
    reads back exactly on the host, and every malformed variant is refused
    with LBM_ERR_ARG before any device work."""
    rng = np.random.default_rng(3)
    p = rng.standard_normal(lbm.lbm_mlp_param_count()).astype(np.float32)
    st = rng.standard_normal(32).astype(np.float32)
    path = tmp_path / "net.bin"
    lbm.write_learned_closure(str(path), p, st)
    assert path.stat().st_size == 8 + 8 + 4 * (p.size + 32)
    p2, st2 = lbm.lbm_read_learned_closure(str(path))
    assert np.array_equal(p2, p) and np.array_equal(st2, st)
    raw = path.read_bytes()
    pp, ss = np.empty(p.size, np.float32), np.empty(32, np.float32)

    def rc_of(data, nparam=p.size, nstats=32):
        q = tmp_path / "bad.bin"
        q.write_bytes(data)
        return lbm.LIB.lbm_read_learned_closure(str(q).encode(), lbm._fp(pp), nparam, lbm._fp(ss), nstats)

    assert rc_of(raw) == lbm.LBM_OK
    assert rc_of(b"LBMMLP02" + raw[8:]) == lbm.LBM_ERR_ARG
    assert "magic" in lbm.lbm_last_error()
    assert rc_of(raw[:8] + np.array([p.size - 1, 32], dtype="<i4").tobytes() + raw[16:]) == lbm.LBM_ERR_ARG
    assert rc_of(raw[:-4]) == lbm.LBM_ERR_ARG
    assert rc_of(raw + b"\0") == lbm.LBM_ERR_ARG
    assert rc_of(raw, nparam=p.size - 1) == lbm.LBM_ERR_ARG
    assert rc_of(raw, nstats=31) == lbm.LBM_ERR_ARG
    assert lbm.LIB.lbm_read_learned_closure(str(tmp_path / "missing.bin").encode(), lbm._fp(pp), p.size,
                                            lbm._fp(ss), 32) == lbm.LBM_ERR_ARG
    assert lbm.LIB.lbm_read_learned_closure(None, lbm._fp(pp), p.size, lbm._fp(ss), 32) == lbm.LBM_ERR_ARG
    assert lbm.LIB.lbm_set_learned_closure_file(None, str(path).encode()) == lbm.LBM_ERR_ARG


def test_committed_network_file_matches_npz(lbm):
    """The trained network ships in both forms; the file form holds the same
    FP32 parameters and statistics as the npz."""
    data = os.path.join(ROOT, "paper_2605_19796_gb300", "data")
    d = np.load(os.path.join(data, "learned_closure.npz"))
    p, st = lbm.lbm_read_learned_closure(os.path.join(data, "learned_closure.bin"))
    assert np.array_equal(p, d["params"].astype(np.float32))
    assert np.array_equal(st, d["stats"].astype(np.float32))


def test_plain_c_program_uses_the_abi(lbm, tmp_path):
    """include/lbm.h is plain C99 (pedantic, no warnings), and a C program
    built against it and linked to the library calls entry points that need
    no device: the ABI version, the default configuration, and an argument
    error with its message."""
    import shutil
    import subprocess

    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_lbm.c"
    src.write_text(
        '#include <stdio.h>\n#include "lbm.h"\n'
        "int main(void) {\n"
        "    lbm_config cfg;\n"
        "    lbm_config_default(&cfg);\n"
        "    int rc = lbm_create(NULL, NULL);\n"
        '    printf("%d %d %d %.3f %d %s\\n", lbm_abi_version(), cfg.lattice, cfg.closure, cfg.c_nu, rc,\n'
        "           lbm_last_error());\n"
        "    return 0;\n"
        "}\n")
    libdir = os.path.join(ROOT, "paper_2605_19796_gb300", "csrc")
    exe = tmp_path / "use_lbm"
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", str(src), "-I",
                    os.path.join(ROOT, "include"), "-L", libdir, "-llbm", "-Wl,-rpath," + libdir, "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split(maxsplit=5)
    assert int(out[0]) == lbm.LIB.lbm_abi_version()
    assert int(out[1]) == 27 and int(out[2]) == lbm.CLOSURES["kcmp"] and float(out[3]) == 0.035
    assert int(out[4]) == lbm.LBM_ERR_ARG and len(out) == 6
