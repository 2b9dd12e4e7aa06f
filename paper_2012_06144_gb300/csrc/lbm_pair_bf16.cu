// lbm_pair_bf16.cu -- instances of the two-cell fused step for BF16 storage of
// the moving populations with the D3Q15 phase lattice (lbm_pair_launch.cuh).
#include "lbm_pair_launch.cuh"

namespace lbm {
namespace pairstep {

cudaError_t launch_pair_bf16(const Params &p, const Storage &sto, int q_hydro, bool g_sw, bool h_sw,
                             const float *phi_in, float *phi_out, int *flag, cudaStream_t st) {
    return launch_pair_layouts<__nv_bfloat16, 15>(p, sto, q_hydro, g_sw, h_sw, phi_in, phi_out, flag, st);
}

}  // namespace pairstep
}  // namespace lbm
