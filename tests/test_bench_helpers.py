"""Host-side pieces of bench.py that the reported numbers depend on."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1104_5432_gb300 import csrc_info  # noqa: E402


def test_kernel_hash_is_path_free_and_covers_flags(monkeypatch):
    from paper_1104_5432_gb300 import build as b
    h = bench.phase_kernel_hash()
    assert len(h) == 16
    # another checkout location gives the same key
    monkeypatch.setattr(b, "INCLUDE", "/elsewhere/include")
    monkeypatch.setattr(b, "CSRC", "/elsewhere/csrc")
    assert bench.phase_kernel_hash() == h
    # other compile flags for the phase-kernel units give another key
    units = [(n, d, ()) for n, d, _ in b.SHAPE_UNITS]
    monkeypatch.setattr(b, "SHAPE_UNITS", units)
    assert bench.phase_kernel_hash() != h


def test_profile_record_is_current_and_complete():
    """The committed ncu record matches the current kernel sources and flags,
    so the bench reports its traffic, instruction and flop counts."""
    rec = json.load(open(os.path.join(ROOT, "profiles", "heatbath_phase_traffic.json")))
    h = bench.phase_kernel_hash()
    for key in ("f32_64^4", "f32_128^4_slab", "f64_64^4"):
        assert "ncu" in rec[key]["captured"] and "--clock-control none" in rec[key]["captured"]
        if rec[key]["source_sha256_16"] != h:
            pytest.skip("the ncu record predates the current phase-kernel sources or flags "
                        "(bench.py then reports traffic as null): retake it")
    f32 = rec["f32_64^4"]
    # DRAM traffic within 20% of the algorithmic 128 B per update
    assert 1.0 <= f32["dram_bytes_per_launch_full_size"] / f32["algorithmic_bytes_per_launch"] < 1.2
    assert bench.recorded_traffic("f32_64^4") == f32["dram_bytes_per_launch_full_size"]
    assert 0 < bench.recorded_traffic("f32_64^4", "warp_inst_per_launch")
    assert 400 < bench.recorded_traffic("f64_64^4", "fp64_flops_per_update") < 1000
    assert 0 <= f32["launch_shape"] < len(csrc_info._F32)


def test_launch_shape_names():
    names = csrc_info.launch_shapes(False)
    assert len(names) == len(csrc_info._F32) == 14
    assert "retry queue" in names[8] and "y-slab" in names[13]
    assert "retry queue" not in names[0]


def test_oracle_all_cores_leg_small():
    """The all-cores oracle leg on a tiny lattice: spawned processes, one
    aggregate rate over the common window."""
    r = bench.oracle_all_cores(4, 4)
    assert r is not None
    ups, n, updates, dt = r
    assert n >= 1 and updates == n * (4 ** 4 // 2) and ups > 0 and dt > 0
