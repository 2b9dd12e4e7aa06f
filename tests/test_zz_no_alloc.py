"""The allocation-free diagnostics entry point, lbm_reduce_state_noalloc.

Some users of this library cannot allocate device memory where they want the
diagnostics: the memory pool of their host application already holds the GPU's
free memory, or their time loop cannot take the synchronisation that cudaMalloc
and cudaFree may cause.  The entry point made for them computes the lbm_reduce
quantities from a state they already hold, with its scratch space in a fixed
array inside the library.  These tests call it through the C ABI and check it
against lbm_reduce on the same state, on two calls in a row (the second call
finds the first call's partial sums still in the shared array), and that the
second call takes no further device memory.  This file is collected last.
"""
import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def lbm():
    from paper_2012_06144_gb300 import _build, lbm

    _build.build()
    lbm.load()
    return lbm


def _close(a, b):
    # same per-cell values; the FP64 sums only differ in their order (momentum
    # sums cancel to ~1e-9, hence the small absolute term)
    for k, (x, y) in enumerate(zip(a, b)):
        assert abs(x - y) <= 1e-9 * abs(y) + 1e-13, (k, x, y)


@pytest.mark.gpu
def test_noalloc_matches_lbm_reduce_twice(lbm):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    prob, phi0 = W.rising_bubble(24, 48, 20, D=12.0, t_ref=1000.0)
    dom, prm = lbm.from_problem(prob)
    sim = lbm.Simulation.from_problem(prob)
    stream = sim.stream.cuda_stream
    sim.init_phase(phi0)

    sim.step(25)
    ref1 = lbm.lbm_reduce(sim.handle)
    _, g1, phi1 = sim.get_state(on_device=True)
    sim.step(10)
    ref2 = lbm.lbm_reduce(sim.handle)
    _, g2, phi2 = sim.get_state(on_device=True)
    torch.cuda.synchronize()

    first = lbm.lbm_reduce_state_noalloc(dom, prm, g1.data_ptr(), phi1.data_ptr(), stream)
    free_before = torch.cuda.mem_get_info()[0]
    second = lbm.lbm_reduce_state_noalloc(dom, prm, g2.data_ptr(), phi2.data_ptr(), stream)
    free_after = torch.cuda.mem_get_info()[0]

    _close(first, ref1)
    _close(second, ref2)
    assert not np.allclose(ref1, ref2)  # the two calls really saw different states
    assert free_after == free_before
    sim.close()


def test_noalloc_rejects_oversized_box(lbm):
    """Boxes beyond the fixed scratch (512^3 cells) are refused before any launch."""
    dom = lbm.make_domain(1024, 512, 512, q_hydro=27)
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_reduce_state_noalloc(dom, lbm.make_params(), 256, 256)
    assert ei.value.status == lbm.LBM_ERR_ARG
    assert "512^3" in lbm.lbm_last_error(None)
