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


class _FakeRates:
    """Stand-in for the throughput probes: fixed rates, no GPU."""
    F64 = 1
    (PROBE_LOG, PROBE_COSPI, PROBE_SINCOSPI, PROBE_SQRT, PROBE_RSQRT, PROBE_LN_TABLE,
     PROBE_COS_TABLE, PROBE_SINCOS_TABLE) = range(8)

    @staticmethod
    def probe_fma_rate(dtype):
        return 5e11  # DFMA/s

    @staticmethod
    def probe_special_rate(fn):
        return 1e10 * (fn + 1)


def test_fp64_roofline_follows_the_algorithmic_model():
    """T_roof = (420 + 10 t) / (2 x DFMA rate) + sum_f n_f / rate_f with the
    update's math-function calls (per trial 2 log + 1 cospi; 2 rsqrt,
    2 sqrt, 1 sincospi); frac = achieved x T_roof.  The logarithm, cosine
    and sine + cosine rates are those of the kernels' own table-driven
    routines (probe ids 5, 6, 7)."""
    t = 1.04
    r = bench.fp64_roofline(_FakeRates, 1.2e9, t)
    T = ((420 + 10 * t) / 1e12 + 2 * t / 6e10 + t / 7e10 + 1 / 8e10 + 2 / 4e10 + 2 / 5e10)
    assert r["peak"] == pytest.approx(1 / T, rel=1e-12)
    assert r["frac"] == pytest.approx(1.2e9 * T, abs=1e-4)
    assert r["algorithmic_flops_per_update"] == pytest.approx(430.4)
    assert r["bound"] == "alu" and r["unit"] == bench.UNIT


def test_summary_is_short_and_last():
    """The summary carries the companion arms in few characters, so the end
    of the bench line (what a truncated log keeps) shows them."""
    arms = {"fp64_plain": {"value": 1.22e9, "roofline": {"frac": 0.61}},
            "fp32_batched": {"value": 3.87e10}, "fp32_temperature_scan": {"value": 3.48e10},
            "fp32_128^4": {"value": 3.92e10}, "fp64_8^4_beta2.3": {"value": 7.0e7},
            "fp32_32^4_beta6.0": {"value": 3.1e10}, "fp64_32^4_beta6.0": {"value": 1.1e9},
            "fp32_over_fp64_plain": 32.8,
            "fp32_vs_fp64_plaquette": {"diff_in_sigma": 0.66},
            "size_sweep_beta6": {"per_size": {f"{n}^4": {"fp32": 1.0, "fp64": 0.1}
                                              for n in (8, 12, 16, 24, 32, 48, 64)}}}
    line = {"value": 4.02e10, "roofline": {"frac": 0.779}, "e2e": {"value": 3.91e10},
            "arms": arms}
    s = bench.summary(line)
    assert s["fp32_batched"] == 38.7 and s["fp64_plain_frac_alu"] == 0.61
    assert len(json.dumps(s)) < 1000
    # both arms print the same config
    assert bench.main_config(1) == bench.main_config(1)
    assert "one checkerboard phase" in bench.main_config(1)["reference_step"]
