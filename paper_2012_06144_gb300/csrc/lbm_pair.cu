// lbm_pair.cu -- the fused coupled step with two cells per thread: the
// single-simulation kernel and its launchers.  The device code, and what the
// form does, are in lbm_pair_impl.cuh.
#include "lbm_pair_impl.cuh"

#ifndef LBM_PAIR_MIN_BLOCKS_WIDE
#define LBM_PAIR_MIN_BLOCKS_WIDE 3  // the same for pairs of lattices holding 46 or more populations
#endif

namespace lbm {
namespace pairstep {

template <int QG, int QP>
constexpr int pair_min_blocks() { return QG + QP >= 46 ? LBM_PAIR_MIN_BLOCKS_WIDE : LBM_PAIR_MIN_BLOCKS; }

template <typename T, int QG, int QP, bool G_SW, bool H_SW>
__global__ void __launch_bounds__(TX *TY *TZ, pair_min_blocks<QG, QP>())
    pair_step_kernel(Params p, Lat<T> lh, Lat<T> lg, const float *__restrict__ phi_in, float *__restrict__ phi_out,
                     int *__restrict__ flag) {
    __shared__ __align__(16) float tile[TZ + 2][TY + 2][ROW];
    // blockIdx.x runs over the (x, y) tiles, x fastest; blockIdx.y over z
    const int nbx = (p.nx + PX - 1) / PX;
    const int by = blockIdx.x / nbx, bx = blockIdx.x - by * nbx;
    pair_tile<T, QG, QP, G_SW, H_SW>(p, lh, lg, phi_in, phi_out, flag, tile, bx, by, blockIdx.y);
}

template <typename T, int QG, int QP, bool G_SW, bool H_SW>
cudaError_t launch_pair(const Params &p, const Storage &sto, const float *pi, float *po, int *flag,
                        cudaStream_t st) {
    const Lat<T> lh{sto.h.rest, static_cast<T *>(sto.h.mov), (unsigned)p.N};
    const Lat<T> lg{sto.g.rest, static_cast<T *>(sto.g.mov), (unsigned)p.N};
    const dim3 block(TX, TY, TZ);
    const dim3 grid(((p.nx + PX - 1) / PX) * ((p.ny + TY - 1) / TY), (p.nz + TZ - 1) / TZ);
    pair_step_kernel<T, QG, QP, G_SW, H_SW><<<grid, block, 0, st>>>(p, lh, lg, pi, po, flag);
    return cudaGetLastError();
}

template <typename T, int QP>
cudaError_t launch_pair_layouts(const Params &p, const Storage &sto, int q_hydro, bool g_sw, bool h_sw,
                                const float *pi, float *po, int *flag, cudaStream_t st) {
    if (g_sw == h_sw) return cudaErrorInvalidValue;
    if (q_hydro == 27)
        return g_sw ? launch_pair<T, 27, QP, true, false>(p, sto, pi, po, flag, st)
                    : launch_pair<T, 27, QP, false, true>(p, sto, pi, po, flag, st);
    if (q_hydro == 19)
        return g_sw ? launch_pair<T, 19, QP, true, false>(p, sto, pi, po, flag, st)
                    : launch_pair<T, 19, QP, false, true>(p, sto, pi, po, flag, st);
    return cudaErrorInvalidValue;
}

}  // namespace pairstep

bool pair_step_applies(const Params &p, int q_hydro, int q_phase, int precision) {
    if (p.step_form == LBM_FORM_FUSED_CELL) return false;
    if (p.step_form != LBM_FORM_FUSED_PAIR && !pair_step_enabled(precision)) return false;
    // the D3Q19 / D3Q27 phase lattices are stored in FP32 (checked on creation)
    const bool qp_ok = q_phase == 15 || ((q_phase == 19 || q_phase == 27) && precision == LBM_PRECISION_FP32);
    return qp_ok && !p.phase_mrt && (q_hydro == 19 || q_hydro == 27) && (p.nx % 2) == 0 &&
           offsets32(p.N, q_hydro, q_phase);
}

cudaError_t launch_pair_step(const Params &p, const Storage &sto, int q_hydro, int q_phase, bool g_sw, bool h_sw,
                             const float *phi_in, float *phi_out, int *flag, cudaStream_t st) {
    if (q_phase != 15) {
        if (sto.precision != LBM_PRECISION_FP32) return cudaErrorInvalidValue;
        if (q_phase == 19)
            return pairstep::launch_pair_layouts<float, 19>(p, sto, q_hydro, g_sw, h_sw, phi_in, phi_out, flag, st);
        if (q_phase == 27)
            return pairstep::launch_pair_layouts<float, 27>(p, sto, q_hydro, g_sw, h_sw, phi_in, phi_out, flag, st);
        return cudaErrorInvalidValue;
    }
    switch (sto.precision) {
        case LBM_PRECISION_FP32:
            return pairstep::launch_pair_layouts<float, 15>(p, sto, q_hydro, g_sw, h_sw, phi_in, phi_out, flag, st);
        case LBM_PRECISION_FP16:
            return pairstep::launch_pair_layouts<__half, 15>(p, sto, q_hydro, g_sw, h_sw, phi_in, phi_out, flag, st);
        case LBM_PRECISION_BF16:
            return pairstep::launch_pair_layouts<__nv_bfloat16, 15>(p, sto, q_hydro, g_sw, h_sw, phi_in, phi_out,
                                                                    flag, st);
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace lbm
