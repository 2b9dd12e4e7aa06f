"""The streaming-pattern probe (the bandwidth ceiling reported next to the
roofline) runs on the GPU and reports every pattern."""
import json
import subprocess

import pytest


@pytest.mark.gpu
def test_pattern_probe_reports_every_pattern():
    from paper_2012_06144_gb300 import _build

    _build.build()
    r = subprocess.run([_build.PROBE, "128", "2"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["n"] == 128 and out["planes"] == 42 and out["unit"] == "GB/s"
    assert "aa_cluster" not in out and "aa_xalign" not in out
    for k in ("copy", "local", "aa_mix", "aa_odd", "pull", "push", "twist", "pair32_g_natural", "pair32_g_swapped",
              "pair16_g_natural", "pair16_g_swapped"):
        assert 0.0 < out[k] < 20000.0, (k, out[k])
