"""Storage precision (weight-shifted FP16 / BF16 vs FP32 vs FP64) on 64^3
decaying HIT, 100 steps, against the FP64-storage GPU run (itself parity-checked
against the oracle).  Bounds (stated here, from the storage mantissas: FP32
24 bits on f, FP16 11 bits and BF16 8 bits on g = f - w, |g| ~ 1e-3):
u rms error vs u_rms = 0.04: FP32 < 1e-6, FP16 < 1e-3 x u_rms, BF16 < 1e-2 x u_rms;
errors ordered FP32 < FP16 < BF16; kinetic energy within 1e-2 (BF16)."""
import pytest

pytestmark = pytest.mark.gpu


def test_storage_precision():
    import torch

    assert torch.cuda.is_available()
    from paper_2605_19796_gb300 import build

    build.build()
    from paper_2605_19796_gb300 import precision

    res = precision.run(n=64, steps=100)
    print(res)
    urms = 0.04
    assert res["fp32"]["u_rms_err"] < 1e-6
    assert res["fp16"]["u_rms_err"] < 1e-3 * urms
    assert res["bf16"]["u_rms_err"] < 1e-2 * urms
    assert res["fp32"]["u_rms_err"] < res["fp16"]["u_rms_err"] < res["bf16"]["u_rms_err"]
    assert res["bf16"]["E_k_rel_err"] < 1e-2
