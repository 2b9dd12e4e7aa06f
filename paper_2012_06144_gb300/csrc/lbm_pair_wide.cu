// lbm_pair_wide.cu -- instances of the two-cell fused step for the other lattice
// pairs of Section 5.1 (FP32 storage): the D3Q19 / D3Q27 phase lattices with D3Q19
// or D3Q27 hydrodynamics, and the two-dimensional D2Q9 pair (lbm_pair_launch.cuh).
#include "lbm_pair_launch.cuh"

namespace lbm {
namespace pairstep {

cudaError_t launch_pair_wide(const Params &p, const Storage &sto, int q_hydro, int q_phase, bool g_sw, bool h_sw,
                             const float *phi_in, float *phi_out, int *flag, cudaStream_t st) {
    if (q_phase == 9) return launch_pair_2d<float>(p, sto, g_sw, h_sw, phi_in, phi_out, flag, st);
    if (q_phase == 19) return launch_pair_layouts<float, 19>(p, sto, q_hydro, g_sw, h_sw, phi_in, phi_out, flag, st);
    if (q_phase == 27) return launch_pair_layouts<float, 27>(p, sto, q_hydro, g_sw, h_sw, phi_in, phi_out, flag, st);
    return cudaErrorInvalidValue;
}

}  // namespace pairstep
}  // namespace lbm
