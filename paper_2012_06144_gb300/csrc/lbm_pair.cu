// lbm_pair.cu -- the fused coupled step with two cells per thread: where it
// applies and which instance runs.  The device code, and what the form does, are
// in lbm_pair_impl.cuh; the kernel and its launch templates in lbm_pair_launch.cuh,
// instantiated per storage format in lbm_pair_fp32.cu, lbm_pair_fp16.cu,
// lbm_pair_bf16.cu and lbm_pair_wide.cu.
#include "lbm_pair_launch.cuh"

namespace lbm {

bool pair_step_applies(const Params &p, int q_hydro, int q_phase, int precision) {
    if (p.step_form == LBM_FORM_FUSED_CELL) return false;
    if (p.step_form != LBM_FORM_FUSED_PAIR && !pair_step_enabled(precision)) return false;
    // the D3Q19 / D3Q27 phase lattices and the D2Q9 pair are stored in FP32
    // (checked on creation)
    const bool f32 = precision == LBM_PRECISION_FP32;
    const bool lat_ok = (q_phase == 15 && (q_hydro == 19 || q_hydro == 27)) ||
                        ((q_phase == 19 || q_phase == 27) && (q_hydro == 19 || q_hydro == 27) && f32) ||
                        (q_phase == 9 && q_hydro == 9 && f32);
    // the MRT phase collision: FP32 storage with the D3Q15 phase lattice; plane
    // offsets beyond 32 bits: FP32 storage with the D3Q15 phase lattice (64-bit offsets)
    const bool coll_ok = !p.phase_mrt || (f32 && q_phase == 15);
    const bool size_ok = offsets32(p.N, q_hydro, q_phase) || (f32 && q_phase == 15);
    return lat_ok && coll_ok && size_ok && (p.nx % 2) == 0;
}

cudaError_t launch_pair_step(const Params &p, const Storage &sto, int q_hydro, int q_phase, bool g_sw, bool h_sw,
                             const float *phi_in, float *phi_out, int *flag, cudaStream_t st) {
    if (q_phase != 15) {
        if (sto.precision != LBM_PRECISION_FP32) return cudaErrorInvalidValue;
        return pairstep::launch_pair_wide(p, sto, q_hydro, q_phase, g_sw, h_sw, phi_in, phi_out, flag, st);
    }
    switch (sto.precision) {
        case LBM_PRECISION_FP32:
            return pairstep::launch_pair_fp32(p, sto, q_hydro, g_sw, h_sw, phi_in, phi_out, flag, st);
        case LBM_PRECISION_FP16:
            return pairstep::launch_pair_fp16(p, sto, q_hydro, g_sw, h_sw, phi_in, phi_out, flag, st);
        case LBM_PRECISION_BF16:
            return pairstep::launch_pair_bf16(p, sto, q_hydro, g_sw, h_sw, phi_in, phi_out, flag, st);
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace lbm
