"""lbm_diagnostics_noalloc: the allocation-free diagnostics entry point, for
callers that cannot allocate device memory (all device memory owned by another
allocator, or no implicit synchronisation from cudaMalloc/cudaFree allowed).

Called through the C ABI on a solver's own population buffer and checked
against the allocating lbm_diagnostics, twice in a row (the static scratch is
shared between calls).  Tolerance: both compute the same FP64 sums from the same
stored populations, in a different summation order: 1e-12 relative (mass,
E_k, enstrophy, max |u|), momentum sums against mass * max |u|.  This file is
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
]


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


def test_noalloc_rejects_too_many_planes(lbm):
    import torch

    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_diagnostics_noalloc(out.data_ptr(), 27, lbm.LBM_FP32, 4, 4, 4097, out_ptr=out.data_ptr())
    assert ei.value.code == lbm.LBM_ERR_ARG
    assert "4096" in lbm.lbm_last_error()
