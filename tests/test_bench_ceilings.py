"""Host logic of the benchmark's pattern ceilings (no GPU): the two-cell step
alternates its two AA layouts, so a step pair's ceiling is the harmonic mean of
the two layouts' bandwidths, and a form's fraction is its algorithmic GB/s over
that mean."""
import json
import types

import pytest

import bench

PROBE = {"n": 512, "planes": 42, "iters": 20, "unit": "GB/s", "copy": 6660.0, "local": 6856.0, "aa_mix": 6579.0,
         "aa_odd": 4431.0, "pull": 6933.0, "push": 6014.0, "twist": 6393.0, "pair32_g_natural": 6978.0,
         "pair32_g_swapped": 6811.0, "pair16_g_natural": 6158.0, "pair16_g_swapped": 5130.0}


def test_two_cell_fp32_ceiling_is_the_harmonic_mean(monkeypatch):
    monkeypatch.setattr(bench.subprocess, "run",
                        lambda *a, **k: types.SimpleNamespace(stdout=json.dumps(PROBE) + "\n", returncode=0))
    c = bench.pattern_ceiling(512, 6800.0)
    hm = 2.0 / (1.0 / 6978.0 + 1.0 / 6811.0)
    assert c["gbs"] == pytest.approx(hm)
    assert c["frac"] == pytest.approx(6800.0 / hm)
    assert c["aa_one_cell_gbs"] == 6579.0
    # a step pair at the ceiling moves 2 x 344 B per cell in 344/6978 + 344/6811 ns-units
    assert 2 * 344 / (344 / 6978.0 + 344 / 6811.0) == pytest.approx(hm)


def test_one_cell_ceiling_when_the_probe_has_no_two_cell_modes(monkeypatch):
    probe = {k: v for k, v in PROBE.items() if not k.startswith("pair")}
    monkeypatch.setattr(bench.subprocess, "run",
                        lambda *a, **k: types.SimpleNamespace(stdout=json.dumps(probe) + "\n", returncode=0))
    c = bench.pattern_ceiling(512, 6000.0)
    assert c["gbs"] == 6579.0 and c["frac"] == pytest.approx(6000.0 / 6579.0)


def test_16bit_ceiling_and_fractions():
    forms = {"fp16": {"value": 23716.0, "bytes_per_cell": 184}, "bf16": {"value": 23468.0, "bytes_per_cell": 184}}
    c = bench.pattern_ceiling_16bit(PROBE, forms)
    hm = 2.0 / (1.0 / 6158.0 + 1.0 / 5130.0)
    assert c["gbs"] == pytest.approx(hm)
    assert c["fp16_frac"] == pytest.approx(23716.0 * 184 / 1e3 / hm)
    assert c["bf16_frac"] == pytest.approx(23468.0 * 184 / 1e3 / hm)
    assert bench.pattern_ceiling_16bit(None, forms) is None
    assert bench.pattern_ceiling_16bit({"copy": 1.0}, forms) is None


def test_ceiling_skipped_for_sizes_the_probe_does_not_take():
    assert bench.pattern_ceiling(48, 1.0) is None
    assert bench.pattern_ceiling(1024, 1.0) is None
