// lbm_pair_fp32.cu -- instances of the two-cell fused step for FP32 storage with
// the D3Q15 phase lattice: SRT or MRT phase collision, 32- or 64-bit plane offsets
// (lbm_pair_launch.cuh).
#include "lbm_pair_launch.cuh"

namespace lbm {
namespace pairstep {

cudaError_t launch_pair_fp32(const Params &p, const Storage &sto, int q_hydro, bool g_sw, bool h_sw,
                             const float *phi_in, float *phi_out, int *flag, cudaStream_t st) {
    if (!offsets32(p.N, q_hydro, 15))
        return p.phase_mrt ? launch_pair_layouts<float, 15, true, true>(p, sto, q_hydro, g_sw, h_sw, phi_in, phi_out,
                                                                        flag, st)
                           : launch_pair_layouts<float, 15, false, true>(p, sto, q_hydro, g_sw, h_sw, phi_in, phi_out,
                                                                         flag, st);
    if (p.phase_mrt)
        return launch_pair_layouts<float, 15, true>(p, sto, q_hydro, g_sw, h_sw, phi_in, phi_out, flag, st);
    return launch_pair_layouts<float, 15>(p, sto, q_hydro, g_sw, h_sw, phi_in, phi_out, flag, st);
}

}  // namespace pairstep
}  // namespace lbm
