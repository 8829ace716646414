"""lbm_diagnostics_noalloc: the allocation-free diagnostics entry point, for
callers that cannot allocate device memory (all device memory owned by another
allocator, or no implicit synchronisation from cudaMalloc/cudaFree allowed).

Called through the C ABI on a solver's own population buffer and checked
against the allocating lbm_diagnostics, twice in a row (the static scratch is
shared between calls).  Tolerance: both compute the same FP64 sums from the same
stored populations, in a different summation order: 1e-12 relative (mass,
E_k, enstrophy, max |u|), momentum sums against mass * max |u|.  Covered: all
four storage formats (the 16-bit ones re-add the lattice weight to the stored
f - w), D3Q19 and D3Q27, walls with a body force, and the second box of a
two-box buffer addressed at its offset b*q*nx*ny*nz elements.  That a call
allocates nothing is checked by the device's free memory (cudaMemGetInfo) and
torch's allocator staying unchanged across repeated calls.  This file is
collected last on purpose.
"""
import numpy as np
import pytest

from paper_2605_19796_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2605_19796_gb300 import build

    build.build()
    from paper_2605_19796_gb300 import lbm as _lbm

    return _lbm


def _check(ref, got):
    for k in (0, 4, 5, 7):
        assert abs(got[k] - ref[k]) <= 1e-12 * abs(ref[k]), (k, got[k], ref[k])
    for k in (1, 2, 3):
        assert abs(got[k] - ref[k]) <= 1e-12 * ref[0] * ref[7], (k, got[k], ref[k])
    assert got[6] == ref[6] == 0.0


CASES = [
    dict(q=27, storage="fp32", shape=(40, 24, 20), bc=(0, 0, 0), force=(0.0, 0.0, 0.0)),
    dict(q=19, storage="fp64", shape=(17, 12, 9), bc=(0, 0, 0), force=(0.0, 0.0, 0.0)),
    dict(q=27, storage="fp64", shape=(20, 13, 6), bc=(0, 1, 0), force=(2e-5, 0.0, 0.0)),
    dict(q=27, storage="fp16", shape=(40, 24, 20), bc=(0, 0, 0), force=(0.0, 0.0, 0.0)),
    dict(q=27, storage="bf16", shape=(24, 16, 12), bc=(0, 0, 0), force=(0.0, 0.0, 0.0)),
    dict(q=19, storage="fp16", shape=(17, 12, 9), bc=(0, 1, 0), force=(1e-5, 0.0, 0.0)),
]

ELEM = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"q{c['q']}-{c['storage']}-bc{c['bc'][1]}")
def test_noalloc_matches_lbm_diagnostics(lbm, case):
    import torch

    nx, ny, nz = case["shape"]
    rho, u = inputs.hit_fields(0, k0=2.0, urms=0.05, seed=7, shape=case["shape"])
    with lbm.Solver(case["q"], case["shape"], 1e-4, closure="kcmp", storage=case["storage"], bc=case["bc"],
                    force=case["force"]) as s:
        s.init_velocity(rho, u)
        for _ in range(2):
            s.step(3)
            ref = s.diagnostics()
            ptr, _ = s.population_buffer()
            for _call in range(2):  # two calls in a row share the static scratch
                out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
                lbm.lbm_diagnostics_noalloc(ptr, case["q"], lbm.STORAGES[case["storage"]], nx, ny, nz,
                                            bc=case["bc"], force=case["force"], out_ptr=out.data_ptr())
                torch.cuda.synchronize()
                _check(ref, out.cpu().numpy())


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_noalloc_second_box_at_its_offset(lbm, storage):
    """Two boxes of different viscosity in one buffer: the call on each box's
    offset reproduces lbm_diagnostics of that box."""
    import torch

    shape = (24, 16, 10)
    nx, ny, nz = shape
    fields = [inputs.hit_fields(0, k0=2.0, urms=0.05, seed=20 + b, shape=shape) for b in range(2)]
    rho = np.stack([f[0] for f in fields])
    u = np.stack([f[1] for f in fields], axis=1)
    with lbm.Solver(27, shape, np.array([2e-5, 3e-3]), closure="kcmp", storage=storage, nbatch=2) as s:
        s.init_velocity(rho, u)
        s.step(4)
        ptr, _ = s.population_buffer()
        refs = [s.diagnostics(b) for b in range(2)]
        assert abs(refs[0][4] - refs[1][4]) > 1e-3 * refs[0][4]  # the boxes differ
        for b in range(2):
            out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
            off = b * 27 * nx * ny * nz * ELEM[storage]
            lbm.lbm_diagnostics_noalloc(ptr + off, 27, lbm.STORAGES[storage], nx, ny, nz, out_ptr=out.data_ptr())
            torch.cuda.synchronize()
            _check(refs[b], out.cpu().numpy())


def test_noalloc_allocates_nothing(lbm):
    """Repeated calls change neither the device's free memory nor torch's
    allocator statistics (the first call, which may load the kernel's module,
    is made before the baseline is taken)."""
    import torch

    shape = (64, 48, 40)
    nx, ny, nz = shape
    rho, u = inputs.hit_fields(0, k0=2.0, urms=0.05, seed=9, shape=shape)
    with lbm.Solver(27, shape, 1e-4, closure="kcmp", storage="fp32") as s:
        s.init_velocity(rho, u)
        ptr, _ = s.population_buffer()
        outs = [torch.zeros(8, dtype=torch.float64, device="cuda") for _ in range(4)]
        lbm.lbm_diagnostics_noalloc(ptr, 27, lbm.LBM_FP32, nx, ny, nz, out_ptr=outs[0].data_ptr())
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        alloc0, reserved0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
        for k in range(1, 4):
            lbm.lbm_diagnostics_noalloc(ptr, 27, lbm.LBM_FP32, nx, ny, nz, out_ptr=outs[k].data_ptr())
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, (free0, free1)
        assert torch.cuda.memory_allocated() == alloc0 and torch.cuda.memory_reserved() == reserved0
        ref = s.diagnostics()
        for k in range(4):
            _check(ref, outs[k].cpu().numpy())


def test_noalloc_rejects_too_many_planes(lbm):
    import torch

    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_diagnostics_noalloc(out.data_ptr(), 27, lbm.LBM_FP32, 4, 4, 4097, out_ptr=out.data_ptr())
    assert ei.value.code == lbm.LBM_ERR_ARG
    assert "4096" in lbm.lbm_last_error()
