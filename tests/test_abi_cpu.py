"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every function that include/lbm.h declares, sizes the workspace, and
rejects invalid problems with LBM_ERR_ARG before touching CUDA."""
import ctypes
import subprocess

import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def lbm():
    from paper_2012_06144_gb300 import _build, lbm

    _build.build()
    lbm.load()
    return lbm


def test_every_declared_function_is_exported(lbm):
    names = lbm.header_functions()
    assert len(names) >= 12
    lib = lbm.load()
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", lbm.library_path()], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(names) <= exported
    # the binding covers exactly the declared functions
    assert set(names) == set(lbm._SIGNATURES)


def test_struct_layout_matches_header(lbm, tmp_path):
    """sizeof / offsetof of the header's structs, as gcc sees them, match the binding."""
    from paper_2012_06144_gb300 import _build

    fields = {"lbm_domain": [f[0] for f in lbm.lbm_domain._fields_],
              "lbm_params": [f[0] for f in lbm.lbm_params._fields_]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lbm.h"', "int main(void) {"]
    for st, names in fields.items():
        lines.append(f'printf("%zu\\n", sizeof({st}));')
        lines += [f'printf("%zu\\n", offsetof({st}, {n}));' for n in names]
    lines += ["return 0; }"]
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", _build.INCLUDE, str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = []
    for cls in (lbm.lbm_domain, lbm.lbm_params):
        want.append(ctypes.sizeof(cls))
        want += [getattr(cls, f[0]).offset for f in cls._fields_]
    assert got == want


def test_workspace_size(lbm):
    d = lbm.make_domain(32, 32, 32, q_hydro=19)
    n = lbm.lbm_workspace_size(d, lbm.make_params())
    N = 32 ** 3
    assert n >= (15 + 19 + 2) * N * 4
    assert n < (15 + 19 + 2) * N * 4 + 200000
    d27 = lbm.make_domain(512, 512, 512, q_hydro=27)
    n27 = lbm.lbm_workspace_size(d27, lbm.make_params())
    assert n27 >= (15 + 27 + 2) * 512 ** 3 * 4  # 23.6 GB at 512^3


def test_workspace_size_16bit(lbm):
    d = lbm.make_domain(64, 64, 64, q_hydro=27)
    n32 = lbm.lbm_workspace_size(d, lbm.make_params())
    n16 = lbm.lbm_workspace_size(d, lbm.make_params(precision=lbm.LBM_PRECISION_FP16, store_g_scale=4096.0))
    N = 64 ** 3
    # rest planes FP32 (2 x 4 B), moving planes 2 B (14 + 26), two phi planes
    assert n16 >= (2 * 4 + 40 * 2 + 2 * 4) * N and n16 < (2 * 4 + 40 * 2 + 2 * 4) * N + 200000
    assert n16 < 0.6 * n32


@pytest.mark.parametrize("field,value", [
    ("nx", 0), ("ny", -3), ("q_phase", 21), ("q_phase", 9), ("q_hydro", 15), ("q_hydro", 9), ("wall", 2),
])
def test_invalid_domain_rejected(lbm, field, value):
    d = lbm.make_domain(8, 8, 8, q_hydro=19)
    if field == "wall":
        d.wall[1] = value
    else:
        setattr(d, field, value)
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_create(d, lbm.make_params())
    assert ei.value.status == lbm.LBM_ERR_ARG
    assert lbm.lbm_last_error(None)


@pytest.mark.parametrize("field,value", [
    ("rho_H", 0.0), ("rho_ratio", -1.0), ("nu_H", 0.0), ("mu_ratio", 0.0), ("sigma", -1e-4), ("xi", 0.0),
    ("mobility", 0.0), ("rho_ref", float("nan")), ("precision", 7), ("nu_H", float("inf")),
    ("store_g_scale", 3.0), ("store_g_scale", -4.0), ("store_phi_ref", float("inf")), ("clamp_phi", 2),
    ("phase_collision", 2), ("phase_collision", -1), ("kernel_form", 4), ("kernel_form", -1),
])
def test_invalid_params_rejected(lbm, field, value):
    p = lbm.make_params()
    setattr(p, field, value)
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_create(lbm.make_domain(8, 8, 8), p)
    assert ei.value.status == lbm.LBM_ERR_ARG


@pytest.mark.parametrize("dom,prm", [
    (dict(nx=7), {}),  # nx odd: a thread's two cells would straddle rows
    (dict(nx=9, nz=1, q_phase=9, q_hydro=9), {}),
])
def test_pair_form_rejected_where_it_does_not_apply(lbm, dom, prm):
    """The two-cell fused step needs nx even: other problems are refused before
    any launch."""
    args = dict(nx=8, ny=8, nz=8, q_hydro=27, q_phase=15)
    args.update(dom)
    d = lbm.make_domain(args["nx"], args["ny"], args["nz"], q_hydro=args["q_hydro"], q_phase=args["q_phase"])
    p = lbm.make_params(kernel_form=lbm.LBM_FORM_FUSED_PAIR, **prm)
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_create(d, p)
    assert ei.value.status == lbm.LBM_ERR_ARG
    assert "two-cell" in lbm.lbm_last_error(None)


def test_too_many_cells_rejected(lbm):
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_workspace_size(lbm.make_domain(2048, 2048, 1024), lbm.make_params())
    assert ei.value.status == lbm.LBM_ERR_ARG


def test_small_workspace_rejected(lbm):
    d, p = lbm.make_domain(8, 8, 8), lbm.make_params()
    n = lbm.lbm_workspace_size(d, p)
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_create(d, p, 0, 256 * 1024, n - 1)  # fake, never dereferenced: rejected first
    assert ei.value.status == lbm.LBM_ERR_OOM
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_create(d, p, 0, 256 * 1024 + 8, n)
    assert ei.value.status == lbm.LBM_ERR_ARG


def test_null_handle_calls(lbm):
    lib = lbm.load()
    assert lib.lbm_step(None, 1) == lbm.LBM_ERR_ARG
    assert lib.lbm_synchronize(None) == lbm.LBM_ERR_ARG
    assert lib.lbm_steps_done(None) == -1
    assert lib.lbm_get_fields(None, None, None, None, 0) == lbm.LBM_ERR_ARG
    out = np.zeros(12)
    assert lib.lbm_reduce(None, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == lbm.LBM_ERR_ARG
    lib.lbm_destroy(None)


def test_problem_translation(lbm):
    prob, _ = W.static_droplet()
    d, p = lbm.from_problem(prob)
    assert (d.nx, d.ny, d.nz, d.q_hydro, d.q_phase) == (32, 32, 32, 19, 15)
    assert p.rho_ratio == 1000.0 and p.mu_ratio == 100.0 and p.sigma == 1e-4


# ---- batch: sizes and validation are host-only ------------------------------------------------------


def test_batch_workspace_size_sums_members(lbm):
    doms = [lbm.make_domain(32, 32, 32, q_hydro=27), lbm.make_domain(5, 3, 2, q_hydro=27),
            lbm.make_domain(48, 96, 48, q_hydro=27)]
    prms = [lbm.make_params(), lbm.make_params(rho_ratio=10.0), lbm.make_params(sigma=1e-3)]
    total = lbm.lbm_batch_workspace_size(doms, prms)
    each = [lbm.lbm_workspace_size(d, p) for d, p in zip(doms, prms)]
    assert total == sum((n + 255) // 256 * 256 for n in each)


def test_batch_create_rejects_before_cuda(lbm):
    a, b = lbm.make_domain(8, 8, 8, q_hydro=27), lbm.make_domain(8, 8, 8, q_hydro=19)
    p = lbm.make_params()
    cases = [
        ([a, b], [p, p], lbm.LBM_ERR_ARG),  # mixed hydrodynamic lattices
        ([a, a], [p, lbm.make_params(precision=lbm.LBM_PRECISION_BF16)], lbm.LBM_ERR_ARG),  # 16-bit storage
        ([a, lbm.make_domain(0, 8, 8)], [p, p], lbm.LBM_ERR_ARG),  # invalid member
        ([a, a], [p, lbm.make_params(xi=0.0)], lbm.LBM_ERR_ARG),
    ]
    for doms, prms, status in cases:
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_batch_create(doms, prms)
        assert ei.value.status == status
        assert lbm.lbm_last_error(None)
    n = lbm.lbm_batch_workspace_size([a, a], [p, p])
    with pytest.raises(lbm.LBMError) as ei:  # fake workspace, never dereferenced: rejected first
        lbm.lbm_batch_create([a, a], [p, p], 0, 256 * 1024, n - 1)
    assert ei.value.status == lbm.LBM_ERR_OOM
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_batch_create([a, a], [p, p], 0, 256 * 1024 + 16, n)
    assert ei.value.status == lbm.LBM_ERR_ARG


def test_batch_null_handle_calls(lbm):
    lib = lbm.load()
    assert lib.lbm_batch_step(None, 1) == lbm.LBM_ERR_ARG
    assert lib.lbm_batch_tune(None, 1, None, None) == lbm.LBM_ERR_ARG
    assert lib.lbm_batch_synchronize(None) == lbm.LBM_ERR_ARG
    assert lib.lbm_batch_size(None) == 0
    assert lib.lbm_batch_member(None, 0) is None
    assert lib.lbm_batch_last_error(None) == b""
    lib.lbm_batch_destroy(None)


def test_mrt_phase_needs_fp32_storage(lbm):
    d = lbm.make_domain(8, 8, 8)
    for prec in (lbm.LBM_PRECISION_FP16, lbm.LBM_PRECISION_BF16):
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_workspace_size(d, lbm.make_params(precision=prec, phase_collision=lbm.LBM_PHASE_MRT))
        assert ei.value.status == lbm.LBM_ERR_ARG
    assert lbm.lbm_workspace_size(d, lbm.make_params(phase_collision=lbm.LBM_PHASE_MRT)) > 0
    with pytest.raises(lbm.LBMError) as ei:  # batches take the SRT phase collision only
        lbm.lbm_batch_create([d, d], [lbm.make_params(), lbm.make_params(phase_collision=lbm.LBM_PHASE_MRT)])
    assert ei.value.status == lbm.LBM_ERR_ARG


def test_unfused_form_workspace_and_limits(lbm):
    d = lbm.make_domain(16, 8, 4, q_hydro=27)
    fused = lbm.lbm_workspace_size(d, lbm.make_params())
    unfused = lbm.lbm_workspace_size(d, lbm.make_params(kernel_form=lbm.LBM_FORM_UNFUSED))
    N = 16 * 8 * 4
    assert unfused >= fused + (15 + 27 + 3) * N * 4  # second grid of both lattices and the velocity field
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_workspace_size(d, lbm.make_params(precision=lbm.LBM_PRECISION_FP16,
                                                  kernel_form=lbm.LBM_FORM_UNFUSED))
    assert ei.value.status == lbm.LBM_ERR_ARG
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_batch_create([d, d], [lbm.make_params(), lbm.make_params(kernel_form=lbm.LBM_FORM_UNFUSED)])
    assert ei.value.status == lbm.LBM_ERR_ARG


def test_other_phase_lattices_limits(lbm):
    """D3Q19 / D3Q27 phase lattices: FP32 storage, SRT, fused form, single simulations."""
    for qp in (19, 27):
        d = lbm.make_domain(16, 8, 4, q_hydro=27, q_phase=qp)
        n = lbm.lbm_workspace_size(d, lbm.make_params())
        assert n >= (qp + 27 + 2) * 16 * 8 * 4 * 4
        for kw in (dict(precision=lbm.LBM_PRECISION_FP16), dict(phase_collision=lbm.LBM_PHASE_MRT),
                   dict(kernel_form=lbm.LBM_FORM_UNFUSED)):
            with pytest.raises(lbm.LBMError) as ei:
                lbm.lbm_workspace_size(d, lbm.make_params(**kw))
            assert ei.value.status == lbm.LBM_ERR_ARG
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_batch_create([d], [lbm.make_params()])
        assert ei.value.status == lbm.LBM_ERR_ARG



def test_batch_member_beyond_32bit_offsets_rejected(lbm):
    """Batch members are addressed with 32-bit plane offsets: (q_hydro - 1) * cells
    at 2^32 or above is refused before any device allocation."""
    big = lbm.make_domain(640, 640, 416, q_hydro=27)  # 26 * 170.4 M cells > 2^32
    assert 26 * 640 * 640 * 416 >= 2 ** 32
    assert lbm.lbm_workspace_size(big, lbm.make_params()) > 0  # a single simulation takes it
    small = lbm.make_domain(8, 8, 8, q_hydro=27)
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_batch_create([small, big], [lbm.make_params(), lbm.make_params()])
    assert ei.value.status == lbm.LBM_ERR_ARG
    assert "2^32" in str(ei.value)

def test_d2q9_pair_limits(lbm):
    p = lbm.make_params()
    ok = lbm.make_domain(64, 32, 1, q_hydro=9, q_phase=9)
    assert lbm.lbm_workspace_size(ok, p) >= (9 + 9 + 2) * 64 * 32 * 4
    bad = [lbm.make_domain(64, 32, 2, q_hydro=9, q_phase=9),          # nz must be 1
           lbm.make_domain(64, 32, 1, q_hydro=19, q_phase=9),         # a pair
           lbm.make_domain(64, 32, 1, q_hydro=9, q_phase=15),
           lbm.make_domain(64, 32, 1, wall=(0, 0, 1), q_hydro=9, q_phase=9)]
    for d in bad:
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_workspace_size(d, p)
        assert ei.value.status == lbm.LBM_ERR_ARG
    for prm in (lbm.make_params(gravity=(0.0, 0.0, 1e-5)), lbm.make_params(precision=lbm.LBM_PRECISION_FP16)):
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_workspace_size(ok, prm)
        assert ei.value.status == lbm.LBM_ERR_ARG


def test_large_box_limits(lbm):
    """Beyond 32-bit plane offsets FP32 storage with the D3Q15 phase lattice runs
    (SRT or MRT); 16-bit storage and the other phase lattices are refused."""
    d = lbm.make_domain(576, 576, 544, q_hydro=27)
    assert lbm.lbm_workspace_size(d, lbm.make_params()) > 0
    assert lbm.lbm_workspace_size(d, lbm.make_params(phase_collision=lbm.LBM_PHASE_MRT)) > 0
    for kw in (dict(precision=lbm.LBM_PRECISION_FP16), dict(precision=lbm.LBM_PRECISION_BF16)):
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_workspace_size(d, lbm.make_params(**kw))
        assert ei.value.status == lbm.LBM_ERR_ARG
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_workspace_size(lbm.make_domain(576, 576, 544, q_hydro=27, q_phase=27), lbm.make_params())
    assert ei.value.status == lbm.LBM_ERR_ARG


def test_pattern_probe_is_built_and_checks_its_arguments(lbm):
    """build() also makes the stand-alone streaming-pattern probe; it refuses box
    sizes it does not handle before touching CUDA (exit status 2)."""
    import os

    from paper_2012_06144_gb300 import _build

    assert os.access(_build.PROBE, os.X_OK)
    for bad in (["48"], ["1024"], ["16"], ["64", "0"]):
        r = subprocess.run([_build.PROBE] + bad, capture_output=True, text=True, timeout=60)
        assert r.returncode == 2, (bad, r.stderr)


def test_batch_candidate_index_round_trip(lbm):
    """The binding's candidate index matches the C tuner's layout
    (halo * 4 + shape) * 2 + order, over all 16 candidates, and the C entry point
    refuses indices outside 0..15 without touching CUDA."""
    seen = set()
    for i in range(len(lbm.BATCH_HALOS) * len(lbm.BATCH_SHAPES) * len(lbm.BATCH_ORDERS)):
        shape, order, halo = lbm.batch_candidate(i)
        assert lbm.batch_choice(shape, order, halo) == i
        assert i == (lbm.BATCH_HALOS.index(halo) * 4 + lbm.BATCH_SHAPES.index(shape)) * 2 + lbm.BATCH_ORDERS.index(order)
        seen.add((shape, order, halo))
    assert len(seen) == 16 and lbm.batch_tile_name("pair") == "32x4x2/pair"
    lib = lbm.load()
    assert lib.lbm_batch_set_config(None, 0) == lbm.LBM_ERR_ARG
