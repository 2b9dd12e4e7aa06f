"""The bounded mbarrier wait behind the TMA-staged phi tile (tma_bar_wait in
lbm_step_impl.cuh) gives up instead of hanging.  A small program built from the
library's own device helpers waits on a barrier that nothing completes (the
wait must run out and report it) and on one that a thread completes (the wait
must succeed); no copy is in flight in either case, so nothing is left pending
when the block exits."""
import json
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu

SOURCE = r"""
#include <chrono>
#include <cstdio>
#include "lbm_step_impl.cuh"

__global__ void wait_once(int *out, int complete) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) lbm::tma_bar_init(&bar);
    __syncthreads();
    if (complete && threadIdx.x == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(lbm::smem_addr(&bar)) : "memory");
    const bool ok = lbm::tma_bar_wait(&bar);
    atomicAdd(out + (ok ? 0 : 1), 1);
}

int main() {
    int *d = nullptr;
    if (cudaMalloc(&d, 4 * sizeof(int)) != cudaSuccess) return 1;
    int h[4] = {0, 0, 0, 0};
    double ms[2];
    for (int complete = 1; complete >= 0; --complete) {
        cudaMemset(d, 0, 2 * sizeof(int));
        const auto t0 = std::chrono::steady_clock::now();
        wait_once<<<1, 64>>>(d, complete);
        if (cudaDeviceSynchronize() != cudaSuccess) return 2;
        ms[complete] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        cudaMemcpy(h + 2 * complete, d, 2 * sizeof(int), cudaMemcpyDeviceToHost);
    }
    std::printf("{\"done_ok\": %d, \"done_timeout\": %d, \"never_ok\": %d, \"never_timeout\": %d, "
                "\"done_ms\": %.3f, \"never_ms\": %.3f}\n", h[2], h[3], h[0], h[1], ms[1], ms[0]);
    cudaFree(d);
    return 0;
}
"""


def test_mbarrier_wait_is_bounded(tmp_path):
    from paper_2012_06144_gb300 import _build

    src = tmp_path / "bounded_wait.cu"
    src.write_text(SOURCE)
    exe = tmp_path / "bounded_wait"
    subprocess.run([_build.nvcc()] + _build.ARCH + ["-O3", "-std=c++17", "--expt-relaxed-constexpr", "-I", _build.CSRC,
                    "-I", _build.INCLUDE, str(src), "-o", str(exe)], check=True, capture_output=True, timeout=600)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["done_ok"] == 64 and out["done_timeout"] == 0      # a completed phase is seen by every thread
    assert out["never_ok"] == 0 and out["never_timeout"] == 64   # a phase that never completes: every thread gives up
    assert out["never_ms"] < 30_000.0                             # within seconds, not a hang
    os.remove(exe)
