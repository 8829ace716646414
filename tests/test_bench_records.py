"""Host logic of bench.py's roofline records (no GPU): a committed ncu record
(DRAM bytes, FP64 instructions or warp instructions per cell) is used only
when its kernel-source hash and kernel instantiation (variant, tile height)
match the run; otherwise the roofline falls back and reports no traffic."""
import importlib.util
import json
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture()
def bench(tmp_path, monkeypatch):
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    spec.loader.exec_module(mod)
    # a private copy of the tree's kernel sources and records
    csrc = tmp_path / "paper_2605_19796_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in mod.KERNEL_SOURCES:
        shutil.copy(os.path.join(ROOT, "paper_2605_19796_gb300", "csrc", f), csrc / f)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(mod, "ROOT", str(tmp_path))
    return mod, tmp_path


def _write(path, name, entry):
    with open(path / "profiles" / name, "w") as fp:
        json.dump({"w": entry}, fp)


def test_kernel_hash_follows_the_kernel_code_only(bench):
    mod, root = bench
    h0 = mod.kernel_hash()
    assert len(h0) == 16 and h0 == mod.kernel_hash()
    (root / "paper_2605_19796_gb300" / "csrc" / "unrelated.cu").write_text("// not a kernel source\n")
    assert mod.kernel_hash() == h0
    src = root / "paper_2605_19796_gb300" / "csrc" / "lbm_step.cuh"
    with open(src, "a") as fp:
        fp.write("\n// a comment only\n/* and a block comment */\n")
    assert mod.kernel_hash() == h0  # comments and layout do not count
    with open(src, "a") as fp:
        fp.write("\nstatic const int changed_code = 1;\n")
    assert mod.kernel_hash() != h0


def test_records_need_matching_hash_and_launch(bench):
    mod, root = bench
    h = mod.kernel_hash()
    launch = {"variant": 12, "tile_y": 8, "zchunk": 16}
    _write(root, "step_kernel_traffic.json", {"kernel_hash": h, "dram_bytes_per_cell": 217.7,
                                                "launch": {"variant": 12, "tile_y": 8}})
    assert mod.traffic_per_cell("w", launch) == pytest.approx(217.7)
    assert mod.traffic_per_cell("w", dict(launch, zchunk=64)) == pytest.approx(217.7)  # chunking: same kernel
    assert mod.traffic_per_cell("w", dict(launch, variant=13)) is None
    assert mod.traffic_per_cell("w", dict(launch, tile_y=16)) is None
    assert mod.traffic_per_cell("other", launch) is None
    _write(root, "step_kernel_traffic.json", {"kernel_hash": "0" * 16, "dram_bytes_per_cell": 217.7,
                                                "launch": {"variant": 12, "tile_y": 8}})
    assert mod.traffic_per_cell("w", launch) is None

    _write(root, "step_kernel_fp64_ops.json", {"kernel_hash": h, "launch": {"variant": 8, "tile_y": 8},
                                                 "fp64_instructions_per_cell": 566.3, "fp64_flops_per_cell": 734.3})
    assert mod.fp64_ops_per_cell("w", {"variant": 8, "tile_y": 8}) == (pytest.approx(566.3), pytest.approx(734.3))
    assert mod.fp64_ops_per_cell("w", {"variant": 1, "tile_y": 8}) is None

    _write(root, "step_kernel_issue.json", {"kernel_hash": h, "launch": {"variant": 8, "tile_y": 8},
                                              "warp_instructions_per_cell": 32.9, "dram_bytes_per_cell": 107.6})
    assert mod.warp_instructions_per_cell("w", {"variant": 8, "tile_y": 8}) == (pytest.approx(32.9),
                                                                               pytest.approx(107.6))
    assert mod.warp_instructions_per_cell("w", {"variant": 13, "tile_y": 8}) is None


def test_missing_records_give_none(bench):
    mod, _ = bench
    assert mod.traffic_per_cell("w", {"variant": 12, "tile_y": 8}) is None
    assert mod.fp64_ops_per_cell("w", {"variant": 8, "tile_y": 8}) is None
    assert mod.warp_instructions_per_cell("w", {"variant": 8, "tile_y": 8}) is None
