"""The roofline's algorithmic bytes per cell follow the paper's own accounting
(tests/golden/byte_accounting.txt, Section 5.1).  One data-movement model counts
the values a step loads and stores; with the paper's two-kernel design it must
give the printed 19 / 16 and 31 / 30 values and 280 / 488 B (FP64), and with the
fused design of this library (u in registers, phi read once and written once, the
rest populations in FP32) the bytes the benchmark divides by."""
import os

import pytest

import bench

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    rows = {}
    with open(os.path.join(HERE, "golden", "byte_accounting.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                step, loads, stores, nbytes, vb = line.split()
                rows[step] = (int(loads), int(stores), int(nbytes), int(vb))
    return rows


def two_kernel_counts(q_phase: int, q_hydro: int):
    """(loads, stores) of the paper's phase and hydro kernels: populations read and
    written once, u exchanged through memory, phi loaded once per kernel."""
    phase = (q_phase + 3 + 1, q_phase + 1)
    hydro = (q_hydro + 3 + 1, q_hydro + 3)
    return phase, hydro


def fused_bytes(q_phase: int, q_hydro: int, store_bytes: int) -> int:
    """One fused launch: every population read and written once (rest populations
    FP32, moving ones in the storage format), u never stored, phi^{k-1} read once
    and phi^k written once (FP32)."""
    per_direction = (4 + (q_phase - 1) * store_bytes) + (4 + (q_hydro - 1) * store_bytes)
    return 2 * per_direction + 4 + 4


def test_model_reproduces_the_printed_accounting():
    g = _golden()
    phase, hydro = two_kernel_counts(15, 27)
    assert phase == g["phase"][:2] and hydro == g["hydro"][:2]
    for (loads, stores), key in ((phase, "phase"), (hydro, "hydro")):
        assert (loads + stores) * g[key][3] == g[key][2]


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("prec,b", [("fp32", 4), ("fp16", 2), ("bf16", 2)])
def test_benchmark_bytes_are_the_fused_model(q, prec, b):
    assert bench.bytes_per_cell(q, prec) == fused_bytes(15, q, b)


def test_fused_design_moves_less_than_the_paper_design():
    # the benchmark's FP32 figure against the paper's FP64 two-kernel figure at 4 bytes
    (pl, ps), (hl, hs) = two_kernel_counts(15, 27)
    assert bench.bytes_per_cell(27, "fp32") == 344
    assert (pl + ps + hl + hs) * 4 == 384  # u written and read back, phi read twice
    assert bench.bytes_per_cell(27, "fp16") == 184


def _tables():
    rows = []
    with open(os.path.join(HERE, "golden", "roofline_tables.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                gpu, kernel, *v = line.split()
                rows.append((gpu, kernel, *map(float, v)))
    return rows


@pytest.mark.parametrize("row", _tables(), ids=lambda r: f"{r[0]}-{r[1]}")
def test_roofline_arithmetic_reproduces_the_papers_tables(row):
    """The benchmark's ceiling (copy bandwidth / bytes per cell) gives the paper's
    kernel estimates, and measured / estimate its printed ratios, to the printed
    digits; the balances follow B_c = n_b / n_f, B_m = b_s / p_peak, l = min(1, B_m / B_c)."""
    gpu, kernel, b_s, p_peak, n_b, n_f, B_c, B_m, l, est, meas, ratio = row
    ceiling = bench.roofline_mlups(b_s, n_b) / 1e3  # GLUPs
    assert abs(ceiling - est) <= 0.005 + 1e-12
    assert abs(100.0 * meas / ceiling - ratio) < 1.0  # printed as whole percent (truncated or rounded)
    assert abs(n_b / n_f - B_c) <= 0.005 + 1e-12
    assert abs(b_s / (p_peak * 1e3) - B_m) <= 0.005 + 1e-12
    assert abs(min(1.0, (b_s / (p_peak * 1e3)) / (n_b / n_f)) - l) <= 0.012  # the table divides the rounded balances


def test_benchmark_ceiling_of_the_fused_step():
    # 344 B per cell at the measured 6770.5 GB/s copy bandwidth
    assert bench.roofline_mlups(6770.5, 344) == pytest.approx(19681.7, abs=0.1)
