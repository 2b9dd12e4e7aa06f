// lbm_internal.h -- launchers shared between the kernel files and the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "lbm.h"
#include "lbm_device.cuh"

namespace lbm {

// Device memory of one lattice: the FP32 rest plane and q-1 planes of moving
// populations in the storage type selected by Storage::precision.
struct LatticeMem {
    float *rest;
    void *mov;
};

struct Storage {
    int precision;  // LBM_PRECISION_*
    LatticeMem h, g;
};

// Extra buffers of the unfused baseline (FP32, natural layout): post-collision
// populations of both lattices and the stored velocity field (3 planes).
struct Unfused {
    float *h_tmp, *g_tmp, *u;
};

// One time step of the unfused baseline: hydro collision (if hydro), phase
// collision, streaming of h, streaming of g (if hydro), over two grids.
cudaError_t launch_unfused(const Params &p, const Unfused &uf, const Storage &sto, int q_hydro, bool hydro,
                           const float *phi_in, float *phi_out, int *flag, cudaStream_t st);

// True if every moving-plane element offset (q - 1) N of both lattices fits 32
// bits (the fused kernel's default addressing; larger boxes take 64-bit plane
// pointers, with FP32 storage, the SRT phase collision and the D3Q15 phase lattice).
inline bool offsets32(long long N, int q_hydro, int q_phase) {
    const int q = q_hydro > q_phase ? q_hydro : q_phase;
    return (unsigned long long)N * (unsigned long long)(q - 1) < (1ull << 32);
}

// The two-cells-per-thread form of the fused step (lbm_pair.cu): taken where it
// applies (nx even, SRT, the D3Q15 phase lattice -- or D3Q19 / D3Q27 with FP32
// storage -- with D3Q19 / D3Q27 hydrodynamics, 32-bit plane offsets) when the handle asks for it
// (LBM_FORM_FUSED_PAIR) or, with LBM_FORM_FUSED, for the storage formats whose
// bit (1 << precision) is set in LBM_PAIR.
#ifndef LBM_PAIR
#define LBM_PAIR 7  // every storage format (FP32, FP16, BF16)
#endif
inline bool pair_step_enabled(int precision) { return ((LBM_PAIR >> precision) & 1) != 0; }
bool pair_step_applies(const Params &p, int q_hydro, int q_phase, int precision);
cudaError_t launch_pair_step(const Params &p, const Storage &sto, int q_hydro, int q_phase, bool g_swapped,
                             bool h_swapped, const float *phi_in, float *phi_out, int *flag, cudaStream_t st);

// One launch of the fused kernel K_k = hydro(k-1) + phase(k) (hydro = true), or
// the first phase step alone (hydro = false).  g_swapped / h_swapped give the
// current AA layout of each lattice.
cudaError_t launch_step(const Params &p, const Storage &sto, int q_hydro, int q_phase, bool g_swapped,
                        bool h_swapped, bool hydro, const float *phi_in, float *phi_out, int *flag, cudaStream_t st);

// h_i = w_i phi0, g_i = 0 (natural layout).
cudaError_t launch_init(const Params &p, const Storage &sto, int q_hydro, int q_phase, const float *phi0,
                        cudaStream_t st);

// phi, u (three planes), p from (g^t, phi^t); outputs may be null.
cudaError_t launch_fields(const Params &p, const Storage &sto, int q_hydro, bool g_swapped, const float *phi,
                          float *out_phi, float *ux, float *uy, float *uz, float *pr, cudaStream_t st);

// Natural-layout planes [i0, i1) of one lattice (is_h: the phase-field lattice h
// with q = q_phase, else g with q = q_hydro) to/from a dense FP32 buffer.
cudaError_t launch_gather(const Params &p, const Storage &sto, bool is_h, int q, bool swapped, int i0, int i1,
                          float *out, cudaStream_t st);
cudaError_t launch_scatter(const Params &p, const Storage &sto, bool is_h, int q, bool swapped, int i0, int i1,
                           const float *in, cudaStream_t st);

// Diagnostics: LBM_DIAG_COUNT raw sums / max into out (device); scratch holds
// kReduceBlocks * kDiagSlots doubles.
constexpr int kReduceBlocks = 1024;
constexpr int kDiagSlots = 12;
cudaError_t launch_reduce(const Params &p, const Storage &sto, int q_hydro, bool g_swapped, const float *phi,
                          double *scratch, double *out, cudaStream_t st);

// Validates a problem and derives the kernel parameters (defined with the C ABI).
lbm_status prepare_problem(const lbm_domain *dom, const lbm_params *prm, Params *out, std::string *why);
void set_thread_error(const std::string &msg);

}  // namespace lbm
