// lbm_aux.cu -- initialisation, field extraction, state transfer and FP64
// diagnostics for the conservative Allen-Cahn LBM, for every population storage
// type (FP32, FP16, BF16 moving populations; FP32 rest populations).
#include "lbm_internal.h"

namespace lbm {

template <typename T>
static LatView<T> h_view(const Params &p, const Storage &s) {
    return {s.h.rest, static_cast<T *>(s.h.mov), p.N, p.h_ref, 1.0f, 1.0f};
}

template <typename T>
static LatView<T> g_view(const Params &p, const Storage &s) {
    return {s.g.rest, static_cast<T *>(s.g.mov), p.N, 0.0f, p.g_scale, p.g_inv_scale};
}

// Runs F<T> for the storage type of s.
#define LBM_BY_PRECISION(s, ...)                       \
    switch ((s).precision) {                           \
        case LBM_PRECISION_FP32: {                     \
            using T = float;                           \
            __VA_ARGS__;                               \
        } break;                                       \
        case LBM_PRECISION_FP16: {                     \
            using T = __half;                          \
            __VA_ARGS__;                               \
        } break;                                       \
        case LBM_PRECISION_BF16: {                     \
            using T = __nv_bfloat16;                   \
            __VA_ARGS__;                               \
        } break;                                       \
        default:                                       \
            return cudaErrorInvalidValue;              \
    }

static dim3 grid1d(long long N) {
    long long b = (N + 255) / 256;
    if (b > 152LL * 64) b = 152LL * 64;
    return dim3((unsigned)(b > 0 ? b : 1));
}

static dim3 grid3d(const Params &p) { return dim3((p.nx + 31) / 32, (p.ny + 7) / 8, p.nz); }

// ---------------------------------------------------------------------------
// h_i = w_i phi0 (= phi0 Gamma_i at u = 0, Section 3.1), g_i = 0 (p* = 0, u = 0).
template <typename T, int QG, int QP>
__global__ void init_kernel(long long N, const float *__restrict__ phi0, LatView<T> h, LatView<T> g) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const float f = phi0[c];
#pragma unroll
        for (int i = 0; i < QP; ++i) h.template store<QP>(i, i, c, wgt<QP>(i) * f);
#pragma unroll
        for (int i = 0; i < QG; ++i) g.template store<QG>(i, i, c, 0.f);
    }
}

template <typename T, int QP>
static cudaError_t launch_init_q(const Params &p, const Storage &sto, int q, const float *phi0, cudaStream_t st) {
    if (q == 9)
        init_kernel<T, 9, QP><<<grid1d(p.N), 256, 0, st>>>(p.N, phi0, h_view<T>(p, sto), g_view<T>(p, sto));
    else if (q == 19)
        init_kernel<T, 19, QP><<<grid1d(p.N), 256, 0, st>>>(p.N, phi0, h_view<T>(p, sto), g_view<T>(p, sto));
    else if (q == 27)
        init_kernel<T, 27, QP><<<grid1d(p.N), 256, 0, st>>>(p.N, phi0, h_view<T>(p, sto), g_view<T>(p, sto));
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_init(const Params &p, const Storage &sto, int q, int q_phase, const float *phi0, cudaStream_t st) {
    if (q_phase != 15) {  // the other phase lattices run with FP32 storage
        if (sto.precision != LBM_PRECISION_FP32) return cudaErrorInvalidValue;
        if (q_phase == 9) return launch_init_q<float, 9>(p, sto, q, phi0, st);
        if (q_phase == 19) return launch_init_q<float, 19>(p, sto, q, phi0, st);
        if (q_phase == 27) return launch_init_q<float, 27>(p, sto, q, phi0, st);
        return cudaErrorInvalidValue;
    }
    LBM_BY_PRECISION(sto, { return launch_init_q<T, 15>(p, sto, q, phi0, st); })
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Macroscopic fields at time level t from (g^t, phi^t): the hydro-step formulas
// of Section 3.2 evaluated without collision.
template <typename T, int QG, bool G_SW>
__device__ __forceinline__ void load_g(const Params &p, const LatView<T> &g, const Cell &C, float gv[QG]) {
#pragma unroll
    for (int i = 0; i < QG; ++i) {
        int slot, idx;
        pop_src_loc<QG, G_SW>(C, i, slot, idx);
        gv[i] = g.template load<QG>(slot, i, idx);
    }
}

template <typename T, int QG, bool G_SW>
__global__ void __launch_bounds__(256) fields_kernel(Params p, LatView<T> g, const float *__restrict__ phi,
                                                     float *__restrict__ out_phi, float *__restrict__ ux,
                                                     float *__restrict__ uy, float *__restrict__ uz,
                                                     float *__restrict__ pr) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const Cell C = make_cell(p, x, y, z);
    float nb[27];
    gather_phi(phi, C, nb);
    float gv[QG];
    load_g<T, QG, G_SW>(p, g, C, gv);
    Hydro<QG> H;
    hydro_macro<QG>(p, gv, nb[13], stencil_sums<QG == 9>(nb), H);
    if (out_phi) out_phi[C.c] = nb[13];
    if (ux) ux[C.c] = H.ux;
    if (uy) uy[C.c] = H.uy;
    if (uz) uz[C.c] = H.uz;
    if (pr) pr[C.c] = H.pstar * H.rho * (1.0f / 3.0f);  // p = p* rho c_s^2
}

cudaError_t launch_fields(const Params &p, const Storage &sto, int q, bool gsw, const float *phi, float *out_phi,
                          float *ux, float *uy, float *uz, float *pr, cudaStream_t st) {
    const dim3 b(32, 8, 1), gr = grid3d(p);
    LBM_BY_PRECISION(sto, {
        const LatView<T> g = g_view<T>(p, sto);
        if (q == 9 && gsw)
            fields_kernel<T, 9, true><<<gr, b, 0, st>>>(p, g, phi, out_phi, ux, uy, uz, pr);
        else if (q == 9)
            fields_kernel<T, 9, false><<<gr, b, 0, st>>>(p, g, phi, out_phi, ux, uy, uz, pr);
        else if (q == 19 && gsw)
            fields_kernel<T, 19, true><<<gr, b, 0, st>>>(p, g, phi, out_phi, ux, uy, uz, pr);
        else if (q == 19)
            fields_kernel<T, 19, false><<<gr, b, 0, st>>>(p, g, phi, out_phi, ux, uy, uz, pr);
        else if (q == 27 && gsw)
            fields_kernel<T, 27, true><<<gr, b, 0, st>>>(p, g, phi, out_phi, ux, uy, uz, pr);
        else if (q == 27)
            fields_kernel<T, 27, false><<<gr, b, 0, st>>>(p, g, phi, out_phi, ux, uy, uz, pr);
        else
            return cudaErrorInvalidValue;
    })
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// State transfer between the in-place AA storage and dense natural FP32 planes.
template <typename T, int Q, bool SW>
__global__ void gather_kernel(Params p, LatView<T> A, int i0, int i1, float *__restrict__ out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const Cell C = make_cell(p, x, y, z);
    for (int i = i0; i < i1; ++i) {
        int slot, idx;
        pop_src_loc<Q, SW>(C, i, slot, idx);
        out[(size_t)(i - i0) * p.N + C.c] = A.template load<Q>(slot, i, idx);
    }
}

template <typename T, int Q, bool SW>
__global__ void scatter_kernel(Params p, LatView<T> A, int i0, int i1, const float *__restrict__ in) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const Cell C = make_cell(p, x, y, z);
    for (int i = i0; i < i1; ++i) {
        int slot, idx;
        pop_src_loc<Q, SW>(C, i, slot, idx);
        A.template store<Q>(slot, i, idx, in[(size_t)(i - i0) * p.N + C.c]);
    }
}

template <typename T, int Q>
static void transfer_q(const Params &p, const LatView<T> &A, bool gather, bool sw, int i0, int i1, float *buf,
                       cudaStream_t st) {
    const dim3 b(32, 8, 1), gr = grid3d(p);
    if (gather) {
        if (sw)
            gather_kernel<T, Q, true><<<gr, b, 0, st>>>(p, A, i0, i1, buf);
        else
            gather_kernel<T, Q, false><<<gr, b, 0, st>>>(p, A, i0, i1, buf);
    } else {
        if (sw)
            scatter_kernel<T, Q, true><<<gr, b, 0, st>>>(p, A, i0, i1, buf);
        else
            scatter_kernel<T, Q, false><<<gr, b, 0, st>>>(p, A, i0, i1, buf);
    }
}

static cudaError_t transfer(const Params &p, const Storage &sto, bool is_h, int q, bool gather, bool sw, int i0,
                            int i1, float *buf, cudaStream_t st) {
    if (i0 < 0 || i1 > q || i0 >= i1) return cudaErrorInvalidValue;
    LBM_BY_PRECISION(sto, {
        const LatView<T> A = is_h ? h_view<T>(p, sto) : g_view<T>(p, sto);
        if (q == 15)
            transfer_q<T, 15>(p, A, gather, sw, i0, i1, buf, st);
        else if (q == 9)
            transfer_q<T, 9>(p, A, gather, sw, i0, i1, buf, st);
        else if (q == 19)
            transfer_q<T, 19>(p, A, gather, sw, i0, i1, buf, st);
        else if (q == 27)
            transfer_q<T, 27>(p, A, gather, sw, i0, i1, buf, st);
        else
            return cudaErrorInvalidValue;
    })
    return cudaGetLastError();
}

cudaError_t launch_gather(const Params &p, const Storage &sto, bool is_h, int q, bool sw, int i0, int i1, float *out,
                          cudaStream_t st) {
    return transfer(p, sto, is_h, q, true, sw, i0, i1, out, st);
}

cudaError_t launch_scatter(const Params &p, const Storage &sto, bool is_h, int q, bool sw, int i0, int i1,
                           const float *in, cudaStream_t st) {
    return transfer(p, sto, is_h, q, false, sw, i0, i1, const_cast<float *>(in), st);
}

// ---------------------------------------------------------------------------
// Diagnostics with FP64 accumulation: a fixed grid of kReduceBlocks blocks, a
// grid-stride loop over cells, warp-shuffle and shared-memory reduction to one
// partial per block, then one block sums the partials in a fixed order (so the
// result is bitwise reproducible).
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

template <typename T, int QG, bool G_SW>
__global__ void __launch_bounds__(256) reduce_partial_kernel(Params p, LatView<T> g, const float *__restrict__ phi,
                                                             double *__restrict__ scratch) {
    double acc[kDiagSlots];
#pragma unroll
    for (int k = 0; k < kDiagSlots; ++k) acc[k] = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < p.N; c += stride) {
        const int x = (int)(c % p.nx);
        const long long r = c / p.nx;
        const int y = (int)(r % p.ny);
        const int z = (int)(r / p.ny);
        const Cell C = make_cell(p, x, y, z);
        float nb[27];
        gather_phi(phi, C, nb);
        float gv[QG];
        load_g<T, QG, G_SW>(p, g, C, gv);
        Hydro<QG> H;
        hydro_macro<QG>(p, gv, nb[13], stencil_sums<QG == 9>(nb), H);
        // bubble indicator: 1 in the light phase, 0 wherever phi >= 1/2
        const double f = nb[13], lf = fmin(fmax(1.0 - 2.0 * f, 0.0), 1.0), rho = H.rho;
        acc[0] += f;
        acc[1] += rho * H.ux;
        acc[2] += rho * H.uy;
        acc[3] += rho * H.uz;
        acc[4] += lf;
        acc[5] += (x + 0.5) * lf;
        acc[6] += (y + 0.5) * lf;
        acc[7] += (z + 0.5) * lf;
        acc[8] += H.ux * lf;
        acc[9] += H.uy * lf;
        acc[10] += H.uz * lf;
        const double um = sqrt((double)H.ux * H.ux + (double)H.uy * H.uy + (double)H.uz * H.uz);
        acc[11] = fmax(acc[11], um);
    }
    __shared__ double sh[8][kDiagSlots];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kDiagSlots; ++k) {
        const double v = (k == 11) ? warp_max(acc[k]) : warp_sum(acc[k]);
        if (lane == 0) sh[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < kDiagSlots) {
        const int k = threadIdx.x;
        double v = sh[0][k];
        for (int w = 1; w < 8; ++w) v = (k == 11) ? fmax(v, sh[w][k]) : v + sh[w][k];
        scratch[(size_t)blockIdx.x * kDiagSlots + k] = v;
    }
}

__global__ void __launch_bounds__(256) reduce_final_kernel(const double *__restrict__ scratch, int nblocks,
                                                           double *__restrict__ out) {
    __shared__ double sh[8][kDiagSlots];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < kDiagSlots; ++k) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
            const double s = scratch[(size_t)b * kDiagSlots + k];
            v = (k == 11) ? fmax(v, s) : v + s;
        }
        v = (k == 11) ? warp_max(v) : warp_sum(v);
        if (lane == 0) sh[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < kDiagSlots) {
        const int k = threadIdx.x;
        double v = sh[0][k];
        for (int w = 1; w < 8; ++w) v = (k == 11) ? fmax(v, sh[w][k]) : v + sh[w][k];
        out[k] = v;
    }
}

cudaError_t launch_reduce(const Params &p, const Storage &sto, int q, bool gsw, const float *phi, double *scratch,
                          double *out, cudaStream_t st) {
    LBM_BY_PRECISION(sto, {
        const LatView<T> g = g_view<T>(p, sto);
        if (q == 9 && gsw)
            reduce_partial_kernel<T, 9, true><<<kReduceBlocks, 256, 0, st>>>(p, g, phi, scratch);
        else if (q == 9)
            reduce_partial_kernel<T, 9, false><<<kReduceBlocks, 256, 0, st>>>(p, g, phi, scratch);
        else if (q == 19 && gsw)
            reduce_partial_kernel<T, 19, true><<<kReduceBlocks, 256, 0, st>>>(p, g, phi, scratch);
        else if (q == 19)
            reduce_partial_kernel<T, 19, false><<<kReduceBlocks, 256, 0, st>>>(p, g, phi, scratch);
        else if (q == 27 && gsw)
            reduce_partial_kernel<T, 27, true><<<kReduceBlocks, 256, 0, st>>>(p, g, phi, scratch);
        else if (q == 27)
            reduce_partial_kernel<T, 27, false><<<kReduceBlocks, 256, 0, st>>>(p, g, phi, scratch);
        else
            return cudaErrorInvalidValue;
    })
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_final_kernel<<<1, 256, 0, st>>>(scratch, kReduceBlocks, out);
    return cudaGetLastError();
}

}  // namespace lbm
