// lbm_pair_launch.cuh -- the single-simulation kernel of the two-cell fused step
// and its launch templates, instantiated per storage format in lbm_pair_fp32.cu,
// lbm_pair_fp16.cu, lbm_pair_bf16.cu and (the other lattice pairs)
// lbm_pair_wide.cu, so that the instances compile in parallel.  The device code,
// and what the form does, are in lbm_pair_impl.cuh; the dispatch in lbm_pair.cu.
#pragma once

#include "lbm_pair_impl.cuh"

#ifndef LBM_PAIR_MIN_BLOCKS_WIDE
#define LBM_PAIR_MIN_BLOCKS_WIDE 3  // the same for pairs of lattices holding 46 or more populations
#endif
#ifndef LBM_PAIR_MIN_BLOCKS_2D
#define LBM_PAIR_MIN_BLOCKS_2D 6  // and for the two-dimensional pair (8192 x 16384, MLUPS: 4 blocks 41,586, 5: 43,991, 6: 45,029, 7: 43,886)
#endif

namespace lbm {
namespace pairstep {

template <int QG, int QP>
constexpr int pair_min_blocks() {
    return QP == 9 ? LBM_PAIR_MIN_BLOCKS_2D : (QG + QP >= 46 ? LBM_PAIR_MIN_BLOCKS_WIDE : LBM_PAIR_MIN_BLOCKS);
}

#ifndef LBM_PAIR_TY2D
#define LBM_PAIR_TY2D 4
#endif

// Tile of the step: 64 x 2 x 2 cells, or 64 x LBM_PAIR_TY2D x 1 for the two-dimensional pair
template <int QP>
constexpr int pair_ty() { return QP == 9 ? LBM_PAIR_TY2D : TY; }
template <int QP>
constexpr int pair_tz() { return QP == 9 ? 1 : TZ; }

// XONLY: tiles that touch only walled x faces test those alone; the instance for
// boxes with x walls (128 x 512 x 128 walled rising bubble: 19,102 against 17,900
// MLUPS; walled 512^3: +0.9 %), while periodic boxes keep the other (the extra path
// costs them 0.5 % through register allocation).
template <typename T, int QG, int QP, bool G_SW, bool H_SW, bool PMRT = false, bool W64 = false, bool XONLY = false>
__global__ void __launch_bounds__(TX *pair_ty<QP>() * pair_tz<QP>(), pair_min_blocks<QG, QP>())
    pair_step_kernel(Params p, Lat<T, W64> lh, Lat<T, W64> lg, const float *__restrict__ phi_in,
                     float *__restrict__ phi_out,
                     int *__restrict__ flag) {
    constexpr int TYk = pair_ty<QP>(), TZk = pair_tz<QP>();
    __shared__ __align__(16) float tile[TZk + 2][TYk + 2][ROW];
    // blockIdx.x runs over the (x, y) tiles, x fastest; blockIdx.y over z
    const int nbx = (p.nx + PX - 1) / PX;
    const int by = blockIdx.x / nbx, bx = blockIdx.x - by * nbx;
    pair_tile<T, QG, QP, G_SW, H_SW, TX, TYk, TZk, XONLY, PMRT>(p, lh, lg, phi_in, phi_out, flag, tile, bx, by,
                                                                blockIdx.y);
}

template <typename T, int QG, int QP, bool G_SW, bool H_SW, bool PMRT = false, bool W64 = false>
cudaError_t launch_pair(const Params &p, const Storage &sto, const float *pi, float *po, int *flag,
                        cudaStream_t st) {
    const Lat<T, W64> lh{sto.h.rest, static_cast<T *>(sto.h.mov), (unsigned)p.N};
    const Lat<T, W64> lg{sto.g.rest, static_cast<T *>(sto.g.mov), (unsigned)p.N};
    constexpr int TYk = pair_ty<QP>(), TZk = pair_tz<QP>();
    const dim3 block(TX, TYk, TZk);
    const dim3 grid(((p.nx + PX - 1) / PX) * ((p.ny + TYk - 1) / TYk), (p.nz + TZk - 1) / TZk);
    if constexpr (QP == 15 && !W64) {
        if (p.wall & 1) {
            pair_step_kernel<T, QG, QP, G_SW, H_SW, PMRT, W64, true><<<grid, block, 0, st>>>(p, lh, lg, pi, po, flag);
            return cudaGetLastError();
        }
    }
    pair_step_kernel<T, QG, QP, G_SW, H_SW, PMRT, W64><<<grid, block, 0, st>>>(p, lh, lg, pi, po, flag);
    return cudaGetLastError();
}

template <typename T, int QP, bool PMRT = false, bool W64 = false>
cudaError_t launch_pair_layouts(const Params &p, const Storage &sto, int q_hydro, bool g_sw, bool h_sw,
                                const float *pi, float *po, int *flag, cudaStream_t st) {
    if (g_sw == h_sw) return cudaErrorInvalidValue;
    if (q_hydro == 27)
        return g_sw ? launch_pair<T, 27, QP, true, false, PMRT, W64>(p, sto, pi, po, flag, st)
                    : launch_pair<T, 27, QP, false, true, PMRT, W64>(p, sto, pi, po, flag, st);
    if (q_hydro == 19)
        return g_sw ? launch_pair<T, 19, QP, true, false, PMRT, W64>(p, sto, pi, po, flag, st)
                    : launch_pair<T, 19, QP, false, true, PMRT, W64>(p, sto, pi, po, flag, st);
    return cudaErrorInvalidValue;
}

// the two-dimensional pair: D2Q9 for both lattices
template <typename T>
cudaError_t launch_pair_2d(const Params &p, const Storage &sto, bool g_sw, bool h_sw, const float *pi, float *po,
                           int *flag, cudaStream_t st) {
    if (g_sw == h_sw) return cudaErrorInvalidValue;
    return g_sw ? launch_pair<T, 9, 9, true, false>(p, sto, pi, po, flag, st)
                : launch_pair<T, 9, 9, false, true>(p, sto, pi, po, flag, st);
}

// Per storage format and lattice pair (each defined in its own file):
// the D3Q15 phase lattice with D3Q19 or D3Q27 hydrodynamics in FP32 (SRT or MRT,
// 32- or 64-bit plane offsets), FP16 and BF16; the D3Q19 / D3Q27 phase lattices
// and the D2Q9 pair in FP32.
cudaError_t launch_pair_fp32(const Params &p, const Storage &sto, int q_hydro, bool g_sw, bool h_sw,
                             const float *phi_in, float *phi_out, int *flag, cudaStream_t st);
cudaError_t launch_pair_fp16(const Params &p, const Storage &sto, int q_hydro, bool g_sw, bool h_sw,
                             const float *phi_in, float *phi_out, int *flag, cudaStream_t st);
cudaError_t launch_pair_bf16(const Params &p, const Storage &sto, int q_hydro, bool g_sw, bool h_sw,
                             const float *phi_in, float *phi_out, int *flag, cudaStream_t st);
cudaError_t launch_pair_wide(const Params &p, const Storage &sto, int q_hydro, int q_phase, bool g_sw, bool h_sw,
                             const float *phi_in, float *phi_out, int *flag, cudaStream_t st);

}  // namespace pairstep
}  // namespace lbm
