// lbm_step.cu -- the fused coupled step of the conservative Allen-Cahn LBM.
//
// One launch K_k advances every cell by the hydrodynamic step k-1 and the
// phase-field step k of Algorithm 2 (arXiv 2012.06144, Section 4.2):
//   hydro(k-1): from g^{k-1}(x) and the stored field phi^{k-1} (27-point
//               neighbourhood): p*, rho, tau, s_nu, F_s, F_p, F_b, F_mu, u_{k-1}
//               (Section 3.2), weighted-orthogonal MRT collision with moment-space
//               forcing (eq:improved_collision), AA streaming of g;
//   phase(k):   phi_k = sum_i h_i^k (eq:updatePhaseField), written to the other
//               phi buffer; normal and theta from phi^{k-1} (eq:interfaceTracking),
//               h^eq = phi_k Gamma_i(u_{k-1}) with u_{k-1} straight from the
//               hydro part in registers, SRT collision (eq:lb_interface), AA
//               streaming of h.
// The same stencil field phi^{k-1} serves both halves, so one pass reads
// q_p h + q g + phi and writes q_p h + q g + phi per cell, and no velocity field is
// stored.  The h lattice runs one time level ahead of g.  The phase-field lattice
// is D3Q15 (the benchmarked pair of Section 5); D3Q19 and D3Q27 give the other
// stencil pairs of Section 5.1 (FP32 storage).
//
// Layout of the work: a block owns a 32 x 2 x 4 tile of cells (one warp = 32
// consecutive x, so every population plane is read and written in full 128-byte
// lines).  The warps first issue the row loads of the phi tile with its one-cell
// halo, then each thread the loads of its q_p + q populations; the tile then goes
// to shared memory, so the stencil values never occupy in-flight registers.  The
// per-tile body lives in lbm_step_impl.cuh, shared with the batched kernel.
// Population addresses are plane base (a kernel parameter) + 4 (X[dx] + Y[dy] +
// Z[dz]), with the per-axis neighbour offsets X, Y, Z computed once per thread
// (periodic wrap folded in); only blocks that touch a walled face evaluate the
// bounce-back conditions.
#include "lbm_step_impl.cuh"

namespace lbm {

constexpr int TY = LBM_TY, TZ = LBM_TZ;

// Resident blocks per SM the register budget is sized for: 4 (64 registers), or 3
// (80 registers) when the two lattices hold 46 populations or more (D3Q27 with D3Q19
// or D3Q27 would spill heavily at 64).
template <int QG, int QP>
constexpr int min_blocks() { return QG + QP >= 46 ? 3 : LBM_MIN_BLOCKS; }

#ifndef LBM_TY2D
#define LBM_TY2D 4  // tile height of the D2Q9 pair (8192 x 16384: 4 gives 3.63, 8 gives 3.72 ms per step)
#endif

// Tile height and depth: 32 x TY x TZ, or 32 x LBM_TY2D x 1 for the D2Q9 pair (one plane).
template <int QP>
constexpr int tile_y() { return QP == 9 ? LBM_TY2D : TY; }
template <int QP>
constexpr int tile_z() { return QP == 9 ? 1 : TZ; }

// L32: population addresses as each lattice's moving-plane base plus a 32-bit
// element offset (s - 1) N + idx (boxes with (q - 1) N < 2^32); otherwise one
// 64-bit base pointer per plane from the kernel parameters.
template <typename T, int QG, int QP, bool G_SW, bool H_SW, bool HYDRO, bool PMRT, bool L32>
__global__ void __launch_bounds__(TX *tile_y<QP>() * tile_z<QP>(), min_blocks<QG, QP>())
    fused_step_kernel(Params p, Planes pl, const float *__restrict__ phi_in, float *__restrict__ phi_out,
                      int *__restrict__ flag) {
    constexpr int TYk = tile_y<QP>(), TZk = tile_z<QP>();
    __shared__ float tile[TZk + 2][TYk + 2][TX + 2];
    // blockIdx.x runs over the (x, y) tiles, x fastest; blockIdx.y over z
    const int nbx = (p.nx + TX - 1) / TX;
    const int by = blockIdx.x / nbx, bx = blockIdx.x - by * nbx;
    if constexpr (L32) {
        const BaseLat32<T> lh{static_cast<float *>(pl.h[0]), static_cast<T *>(pl.h[1]), (unsigned)p.N},
            lg{static_cast<float *>(pl.g[0]), static_cast<T *>(pl.g[1]), (unsigned)p.N};
        tile_update<T, QG, QP, G_SW, H_SW, HYDRO, PMRT, TYk, TZk>(p, lh, lg, phi_in, phi_out, flag, tile, bx, by,
                                                                  blockIdx.y, threadIdx.x, threadIdx.y, threadIdx.z);
    } else {
        tile_update<T, QG, QP, G_SW, H_SW, HYDRO, PMRT, TYk, TZk>(p, TableLat{pl.h}, TableLat{pl.g}, phi_in,
                                                                  phi_out, flag, tile, bx, by, blockIdx.y,
                                                                  threadIdx.x, threadIdx.y, threadIdx.z);
    }
}

template <typename T, int QG, int QP, bool G_SW, bool H_SW, bool HYDRO, bool PMRT, bool L32>
static cudaError_t launch_k(const Params &p, const Planes &pl, const float *pi, float *po, int *flag,
                            cudaStream_t st) {
    constexpr int TYk = tile_y<QP>(), TZk = tile_z<QP>();
    const dim3 block(TX, TYk, TZk);
    const dim3 grid(((p.nx + TX - 1) / TX) * ((p.ny + TYk - 1) / TYk), (p.nz + TZk - 1) / TZk);
    fused_step_kernel<T, QG, QP, G_SW, H_SW, HYDRO, PMRT, L32><<<grid, block, 0, st>>>(p, pl, pi, po, flag);
    return cudaGetLastError();
}

// Addressing per storage type and lattice pair, from a same-GPU comparison on the
// benchmark boxes (32-bit offsets against per-plane pointers, MLUPS): FP32
// D3Q15+D3Q27 +0.6 % (periodic 512^3) and +3.2 % (walled 128x512x128), FP16 +2.7 %,
// D2Q9 +2.4 %; BF16 -0.7 %, D3Q15+D3Q19 -1.0 %, D3Q19+D3Q19 -4.0 %, D3Q27+D3Q27 0.0 %.
#ifndef LBM_ADDR_POLICY
#define LBM_ADDR_POLICY -1  // -1: per configuration (below); 0: pointers everywhere; 1: offsets everywhere
#endif

template <typename T, int QG, int QP>
constexpr bool prefer_offsets32() {
    if (LBM_ADDR_POLICY >= 0) return LBM_ADDR_POLICY == 1 && !(QG == 19 && !std::is_same<T, float>::value);
    if (std::is_same<T, __nv_bfloat16>::value) return false;
    if (QG == 19 || QP == 19 || QP == 27) return false;
    return true;  // D3Q15 + D3Q27 in FP32 or FP16, and D2Q9
}

template <typename T, int QG, int QP, bool G_SW, bool H_SW, bool HYDRO, bool PMRT>
static cudaError_t launch(const Params &p, const Planes &pl, const float *pi, float *po, int *flag,
                          cudaStream_t st) {
    if constexpr (prefer_offsets32<T, QG, QP>()) {
        if (offsets32(p.N, QG, QP)) return launch_k<T, QG, QP, G_SW, H_SW, HYDRO, PMRT, true>(p, pl, pi, po, flag, st);
        // larger boxes: the pointer form, FP32 / D3Q15 only (checked on creation)
        if constexpr (std::is_same<T, float>::value && QP == 15)
            return launch_k<T, QG, QP, G_SW, H_SW, HYDRO, PMRT, false>(p, pl, pi, po, flag, st);
        else
            return cudaErrorInvalidValue;
    } else {
        return launch_k<T, QG, QP, G_SW, H_SW, HYDRO, PMRT, false>(p, pl, pi, po, flag, st);
    }
}


// The layouts of one time step: g natural and h swapped, or g swapped and h
// natural (h runs one AA step ahead); the first phase step alone (no hydro)
// starts from natural h.
template <typename T, int QP, bool PMRT>
static cudaError_t launch_layouts(const Params &p, const Planes &pl, int q_hydro, bool g_sw, bool h_sw, bool hydro,
                                  const float *phi_in, float *phi_out, int *flag, cudaStream_t st) {
    if (!hydro) {
        if (h_sw) return cudaErrorInvalidValue;
        return launch<T, 19, QP, false, false, false, PMRT>(p, pl, phi_in, phi_out, flag, st);
    }
    if (g_sw == h_sw) return cudaErrorInvalidValue;
    if constexpr (QP == 9) {  // the two-dimensional pair: D2Q9 for both lattices
        if (q_hydro != 9) return cudaErrorInvalidValue;
        return g_sw ? launch<T, 9, 9, true, false, true, PMRT>(p, pl, phi_in, phi_out, flag, st)
                    : launch<T, 9, 9, false, true, true, PMRT>(p, pl, phi_in, phi_out, flag, st);
    } else {
        if (q_hydro == 19)
            return g_sw ? launch<T, 19, QP, true, false, true, PMRT>(p, pl, phi_in, phi_out, flag, st)
                        : launch<T, 19, QP, false, true, true, PMRT>(p, pl, phi_in, phi_out, flag, st);
        if (q_hydro == 27)
            return g_sw ? launch<T, 27, QP, true, false, true, PMRT>(p, pl, phi_in, phi_out, flag, st)
                        : launch<T, 27, QP, false, true, true, PMRT>(p, pl, phi_in, phi_out, flag, st);
        return cudaErrorInvalidValue;
    }
}

template <typename T>
static Planes planes_of(const Params &p, const Storage &sto, int q_hydro, int q_phase) {
    Planes pl;
    pl.h[0] = sto.h.rest;
    for (int i = 1; i < 27; ++i) pl.h[i] = i < q_phase ? static_cast<T *>(sto.h.mov) + (size_t)(i - 1) * p.N : nullptr;
    pl.g[0] = sto.g.rest;
    for (int i = 1; i < 27; ++i) pl.g[i] = i < q_hydro ? static_cast<T *>(sto.g.mov) + (size_t)(i - 1) * p.N : nullptr;
    return pl;
}

cudaError_t launch_step(const Params &p, const Storage &sto, int q_hydro, int q_phase, bool g_sw, bool h_sw,
                        bool hydro, const float *phi_in, float *phi_out, int *flag, cudaStream_t st) {
    if (hydro && pair_step_applies(p, q_hydro, q_phase, sto.precision))
        return launch_pair_step(p, sto, q_hydro, q_phase, g_sw, h_sw, phi_in, phi_out, flag, st);
    // the MRT phase collision and the D3Q19 / D3Q27 phase lattices: FP32 storage
    if (p.phase_mrt || q_phase != 15) {
        if (sto.precision != LBM_PRECISION_FP32) return cudaErrorInvalidValue;
        const Planes pl = planes_of<float>(p, sto, q_hydro, q_phase);
        if (p.phase_mrt && q_phase == 15)
            return launch_layouts<float, 15, true>(p, pl, q_hydro, g_sw, h_sw, hydro, phi_in, phi_out, flag, st);
        if (p.phase_mrt) return cudaErrorInvalidValue;
        if (q_phase == 9)
            return launch_layouts<float, 9, false>(p, pl, q_hydro, g_sw, h_sw, hydro, phi_in, phi_out, flag, st);
        if (q_phase == 19)
            return launch_layouts<float, 19, false>(p, pl, q_hydro, g_sw, h_sw, hydro, phi_in, phi_out, flag, st);
        if (q_phase == 27)
            return launch_layouts<float, 27, false>(p, pl, q_hydro, g_sw, h_sw, hydro, phi_in, phi_out, flag, st);
        return cudaErrorInvalidValue;
    }
    switch (sto.precision) {
        case LBM_PRECISION_FP32:
            return launch_layouts<float, 15, false>(p, planes_of<float>(p, sto, q_hydro, 15), q_hydro, g_sw, h_sw,
                                                    hydro, phi_in, phi_out, flag, st);
        case LBM_PRECISION_FP16:
            return launch_layouts<__half, 15, false>(p, planes_of<__half>(p, sto, q_hydro, 15), q_hydro, g_sw, h_sw,
                                                     hydro, phi_in, phi_out, flag, st);
        case LBM_PRECISION_BF16:
            return launch_layouts<__nv_bfloat16, 15, false>(p, planes_of<__nv_bfloat16>(p, sto, q_hydro, 15), q_hydro,
                                                            g_sw, h_sw, hydro, phi_in, phi_out, flag, st);
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace lbm
