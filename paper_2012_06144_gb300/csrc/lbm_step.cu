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
// 15 h + q g + phi and writes 15 h + q g + phi per cell, and no velocity field is
// stored.  The h lattice runs one time level ahead of g.
#include "lbm_internal.h"

namespace lbm {

template <int QG, bool G_SW, bool H_SW, bool HYDRO>
__global__ void __launch_bounds__(256) fused_step_kernel(Params p, float *__restrict__ h, float *__restrict__ g,
                                                         const float *__restrict__ phi_in,
                                                         float *__restrict__ phi_out, int *__restrict__ flag) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const Cell C = make_cell(p, x, y, z);
    const long long N = p.N;

    float nb[27];
    gather_phi(phi_in, C, nb);
    float gv[QG];
    if (HYDRO) {
#pragma unroll
        for (int i = 0; i < QG; ++i) gv[i] = g[pop_src<QG, G_SW>(C, N, i)];
    }
    float hv[15];
#pragma unroll
    for (int i = 0; i < 15; ++i) hv[i] = h[pop_src<15, H_SW>(C, N, i)];

    // ---- hydrodynamic step k-1
    float ux = 0.f, uy = 0.f, uz = 0.f;
    if (HYDRO) {
        Hydro<QG> Hd;
        hydro_macro<QG>(p, gv, nb, Hd);
        const HydroPost<QG> P = hydro_post<QG>(Hd);
        // the rest population takes the remainder of the zeroth moment, so that
        // sum_i g*_i = p* holds to rounding (the FP32 weights do not sum to 1)
        float gsum = 0.f;
#pragma unroll
        for (int i = 1; i < QG; i += 2) {
            float E, O;
            hydro_gstar_pair<QG>(P, i, E, O);
            const float a = E + O, b = E - O;
            g[pop_dst<QG, G_SW>(C, N, i)] = a;
            g[pop_dst<QG, G_SW>(C, N, i + 1)] = b;
            gsum += a + b;
        }
        g[pop_dst<QG, G_SW>(C, N, 0)] = Hd.pstar - gsum;
        ux = Hd.ux;
        uy = Hd.uy;
        uz = Hd.uz;
        if (!(fabsf(Hd.pstar) < 1e30f)) *flag = 1;
    }

    // ---- phase-field step k
    // phi_k = sum_i h_i, accumulated without rounding loss (the collision
    // below puts the remainder of this sum into the rest population, so any
    // rounding here would be a per-cell mass error)
    DFloat phis{hv[0], 0.f};
#pragma unroll
    for (int i = 1; i < 15; ++i) two_sum_acc(phis, hv[i]);
    const float phik = phis.hi + phis.lo;
    phi_out[C.c] = phik;
    if (!(fabsf(phik) < 1e30f)) *flag = 1;

    float Gx, Gy, Gz;
    stencil_grad<15>(nb, Gx, Gy, Gz);
    const float G2 = Gx * Gx + Gy * Gy + Gz * Gz;
    float nx = 0.f, ny = 0.f, nz = 0.f;
    if (G2 > 1e-24f) {
        float inv = rsqrtf(G2);
        inv = inv * (1.5f - 0.5f * G2 * inv * inv);  // one Newton step: no systematic bias in |n|
        nx = Gx * inv;
        ny = Gy * inv;
        nz = Gz * inv;
    }
    const float pc = nb[13] - 0.5f;
    const float theta = (1.0f - 4.0f * pc * pc) * p.inv_xi;
    const float uu = 1.5f * (ux * ux + uy * uy + uz * uz);
    const float om = p.omega_phi, fc = 1.0f - 0.5f * om;
    // h*_i = h_i + omega (h^eq_i - h_i - F_i/2) + F_i over opposite pairs, with
    // h^eq = phi_k w (1 + 3 e.u + 4.5 (e.u)^2 - 1.5 u.u) and F_i = theta w e.n.
    // The non-equilibrium h^eq_i - h_i is formed as fma(phi_hi, w, -h_i) +
    // phi_lo w + phi w (velocity terms), so it carries no rounding of the large
    // product phi w; the rest population takes the remainder so that
    // sum_i h*_i = phi_k holds to the rounding of one store.
    DFloat hsum{0.f, 0.f};
#pragma unroll
    for (int i = 1; i < 15; i += 2) {
        const V3 e = vel<15>(i);
        const float w = wgt<15>(i);
        const float eu = e.x * ux + e.y * uy + e.z * uz;
        const float en = e.x * nx + e.y * ny + e.z * nz;
        const float pw = phik * w;
        const float x_even = pw * (4.5f * eu * eu - uu) + phis.lo * w;
        const float x_odd = pw * 3.0f * eu;
        const float F = fc * (theta * w * en);
        const float neq_a = fmaf(phis.hi, w, -hv[i]) + (x_even + x_odd);
        const float neq_b = fmaf(phis.hi, w, -hv[i + 1]) + (x_even - x_odd);
        const float a = hv[i] + fmaf(om, neq_a, F);
        const float b = hv[i + 1] + fmaf(om, neq_b, -F);
        h[pop_dst<15, H_SW>(C, N, i)] = a;
        h[pop_dst<15, H_SW>(C, N, i + 1)] = b;
        two_sum_acc(hsum, a);
        two_sum_acc(hsum, b);
    }
    h[pop_dst<15, H_SW>(C, N, 0)] = (phis.hi - hsum.hi) + (phis.lo - hsum.lo);
}

template <int QG, bool G_SW, bool H_SW, bool HYDRO>
static cudaError_t launch(const Params &p, float *h, float *g, const float *pi, float *po, int *flag,
                          cudaStream_t st) {
    const dim3 block(32, 8, 1);
    const dim3 grid((p.nx + 31) / 32, (p.ny + 7) / 8, p.nz);
    fused_step_kernel<QG, G_SW, H_SW, HYDRO><<<grid, block, 0, st>>>(p, h, g, pi, po, flag);
    return cudaGetLastError();
}

cudaError_t launch_step(const Params &p, int q_hydro, bool g_sw, bool h_sw, bool hydro, float *h, float *g,
                        const float *phi_in, float *phi_out, int *flag, cudaStream_t st) {
    if (!hydro) {
        if (h_sw) return cudaErrorInvalidValue;  // the first phase step starts from natural h
        return launch<19, false, false, false>(p, h, g, phi_in, phi_out, flag, st);
    }
    if (g_sw == h_sw) return cudaErrorInvalidValue;  // h runs one AA step ahead of g
    if (q_hydro == 19)
        return g_sw ? launch<19, true, false, true>(p, h, g, phi_in, phi_out, flag, st)
                    : launch<19, false, true, true>(p, h, g, phi_in, phi_out, flag, st);
    if (q_hydro == 27)
        return g_sw ? launch<27, true, false, true>(p, h, g, phi_in, phi_out, flag, st)
                    : launch<27, false, true, true>(p, h, g, phi_in, phi_out, flag, st);
    return cudaErrorInvalidValue;
}

}  // namespace lbm
