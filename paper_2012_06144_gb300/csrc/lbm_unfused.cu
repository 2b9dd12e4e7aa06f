// lbm_unfused.cu -- the unfused baseline: the passes of the paper's
// straightforward algorithm (Algorithm 1, Section 4.2) on the GPU.
//
// Per time step four kernels over two grids of natural-layout FP32 populations:
//   hydro_collide  g(x) -> g_tmp(x), stores u      (collision of the velocity PDFs)
//   phase_collide  h(x) -> h_tmp(x), stores phi    (collision of the phase-field PDFs,
//                                                   phi = sum h, eq:updatePhaseField)
//   stream<15>     h_tmp -> h                      (streaming of the phase-field PDFs)
//   stream<q>      g_tmp -> g                      (streaming of the velocity PDFs)
// The update is the fused step's (same time levels: hydro(k-1) then phase(k),
// the hydro half handing u_{k-1} to the phase half, here through a stored field),
// so the same oracle checks both; what differs is the data movement: each
// population crosses HBM three times per step instead of once (at D3Q27,
// 708 B/cell against 344 B/cell), which is the gap the paper's Algorithm 2 closes.
// Kept as the measured baseline of that comparison; not tuned.
#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr int BX = 32, BY = 8;

dim3 grid_of(const Params &p) { return dim3((p.nx + BX - 1) / BX, (p.ny + BY - 1) / BY, p.nz); }

// Collision of the velocity PDFs at each cell (Section 3.2): g^{k-1}(x) and the
// phi^{k-1} neighbourhood give p*, rho, the forces and u_{k-1}; the
// post-collision populations (eq:improved_collision) go to g_tmp at x.
template <int QG>
__global__ void __launch_bounds__(BX *BY) hydro_collide_kernel(Params p, const float *__restrict__ g,
                                                              float *__restrict__ g_tmp,
                                                              const float *__restrict__ phi,
                                                              float *__restrict__ u, int *__restrict__ flag) {
    const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y, z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const Cell C = make_cell(p, x, y, z);
    const size_t N = (size_t)p.N;
    float gv[QG], nb[27];
#pragma unroll
    for (int i = 0; i < QG; ++i) gv[i] = g[i * N + C.c];
    gather_phi(phi, C, nb);
    Hydro<QG> H;
    hydro_macro<QG>(p, gv, nb[13], stencil_sums(nb), H);
    const HydroPost<QG> P = hydro_post<QG>(H);
    float gsum = 0.f;
#pragma unroll
    for (int i = 1; i < QG; i += 2) {
        float E, O;
        hydro_gstar_pair<QG>(P, i, E, O);
        g_tmp[i * N + C.c] = E + O;
        g_tmp[(i + 1) * N + C.c] = E - O;
        gsum += (E + O) + (E - O);
    }
    g_tmp[C.c] = H.pstar - gsum;  // zeroth moment p* kept to rounding
    u[C.c] = H.ux;
    u[N + C.c] = H.uy;
    u[2 * N + C.c] = H.uz;
    if (!(fabsf(H.pstar) < 1e30f)) *flag = 1;
}

// Collision of the phase-field PDFs at each cell (Section 3.1): phi_k = sum h^k,
// normal and theta from the phi^{k-1} neighbourhood, u_{k-1} from the stored
// field; SRT or the MRT of Section 3.1; post-collision populations to h_tmp.
template <bool PMRT>
__global__ void __launch_bounds__(BX *BY) phase_collide_kernel(Params p, const float *__restrict__ h,
                                                              float *__restrict__ h_tmp,
                                                              const float *__restrict__ phi_prev,
                                                              float *__restrict__ phi_next,
                                                              const float *__restrict__ u,
                                                              int *__restrict__ flag) {
    const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y, z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const Cell C = make_cell(p, x, y, z);
    const size_t N = (size_t)p.N;
    float hv[15], nb[27];
#pragma unroll
    for (int i = 0; i < 15; ++i) hv[i] = h[i * N + C.c];
    float phik = hv[0];
#pragma unroll
    for (int i = 1; i < 15; ++i) phik += hv[i];
    phi_next[C.c] = phik;
    if (!(fabsf(phik) < 1e30f)) *flag = 1;
    gather_phi(phi_prev, C, nb);
    float Gx, Gy, Gz;
    stencil_grad<15>(stencil_sums(nb), Gx, Gy, Gz);
    const float G2 = Gx * Gx + Gy * Gy + Gz * Gz;
    float nx = 0.f, ny = 0.f, nz = 0.f;
    if (G2 > 1e-24f) {
        const float inv = 1.0f / sqrtf(G2);
        nx = Gx * inv;
        ny = Gy * inv;
        nz = Gz * inv;
    }
    const float pc = nb[13] - 0.5f;
    const float theta = (1.0f - 4.0f * pc * pc) * p.inv_xi;
    const float ux = u[C.c], uy = u[N + C.c], uz = u[2 * N + C.c];
    const float uu = ux * ux + uy * uy + uz * uz;
    float heq[15], F[15];
#pragma unroll
    for (int i = 0; i < 15; ++i) {
        const V3 e = vel<15>(i);
        const float w = wgt<15>(i);
        const float eu = e.x * ux + e.y * uy + e.z * uz;
        heq[i] = phik * w * (1.0f + 3.0f * eu + 4.5f * eu * eu - 1.5f * uu);  // h^eq = phi Gamma_i
        F[i] = theta * w * (e.x * nx + e.y * ny + e.z * nz);                 // eq:interfaceTracking
    }
    float om = p.omega_phi;
    float cx = 0.f, cy = 0.f, cz = 0.f;
    if constexpr (PMRT) {  // first-order moments with omega_phi, the rest with 1 (weighted basis)
        float Jx = 0.f, Jy = 0.f, Jz = 0.f;
#pragma unroll
        for (int i = 0; i < 15; ++i) {
            const V3 e = vel<15>(i);
            const float d = hv[i] - heq[i] + 0.5f * F[i];
            Jx += e.x * d;
            Jy += e.y * d;
            Jz += e.z * d;
        }
        cx = 3.0f * (1.0f - om) * Jx;
        cy = 3.0f * (1.0f - om) * Jy;
        cz = 3.0f * (1.0f - om) * Jz;
        om = 1.0f;
    }
    float dsum = 0.f;
#pragma unroll
    for (int i = 1; i < 15; ++i) {
        const V3 e = vel<15>(i);
        float hs = hv[i] + om * (heq[i] - hv[i] - 0.5f * F[i]) + F[i];  // eq:lb_interface
        if constexpr (PMRT) hs += wgt<15>(i) * (e.x * cx + e.y * cy + e.z * cz);
        h_tmp[i * N + C.c] = hs;
        dsum += hs - hv[i];
    }
    h_tmp[C.c] = hv[0] - dsum;  // the cell's phase mass kept to rounding
}

// Streaming by pull: f_i(x) = f*_i(x - e_i), or f*_opp(i)(x) when x - e_i lies
// beyond a wall (half-way bounce-back).
template <int Q>
__global__ void __launch_bounds__(BX *BY) stream_kernel(Params p, const float *__restrict__ src,
                                                       float *__restrict__ dst) {
    const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y, z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const Cell C = make_cell(p, x, y, z);
    const size_t N = (size_t)p.N;
    dst[C.c] = src[C.c];
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const V3 e = vel<Q>(i);
        dst[i * N + C.c] = leaves(C, e, -1) ? src[(size_t)opp(i) * N + C.c] : src[i * N + nbr(C, -e.x, -e.y, -e.z)];
    }
}

}  // namespace

cudaError_t launch_unfused(const Params &p, const Unfused &uf, const Storage &sto, int q_hydro, bool hydro,
                           const float *phi_in, float *phi_out, int *flag, cudaStream_t st) {
    if (sto.precision != LBM_PRECISION_FP32) return cudaErrorInvalidValue;
    const dim3 b(BX, BY), gr = grid_of(p);
    float *h = sto.h.rest, *g = sto.g.rest;  // FP32: the moving planes follow the rest plane
    if (hydro) {
        if (q_hydro == 19)
            hydro_collide_kernel<19><<<gr, b, 0, st>>>(p, g, uf.g_tmp, phi_in, uf.u, flag);
        else if (q_hydro == 27)
            hydro_collide_kernel<27><<<gr, b, 0, st>>>(p, g, uf.g_tmp, phi_in, uf.u, flag);
        else
            return cudaErrorInvalidValue;
    }
    if (p.phase_mrt)
        phase_collide_kernel<true><<<gr, b, 0, st>>>(p, h, uf.h_tmp, phi_in, phi_out, uf.u, flag);
    else
        phase_collide_kernel<false><<<gr, b, 0, st>>>(p, h, uf.h_tmp, phi_in, phi_out, uf.u, flag);
    stream_kernel<15><<<gr, b, 0, st>>>(p, uf.h_tmp, h);
    if (hydro) {
        if (q_hydro == 19)
            stream_kernel<19><<<gr, b, 0, st>>>(p, uf.g_tmp, g);
        else
            stream_kernel<27><<<gr, b, 0, st>>>(p, uf.g_tmp, g);
    }
    return cudaGetLastError();
}

}  // namespace lbm
