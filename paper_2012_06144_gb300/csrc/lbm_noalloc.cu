// lbm_noalloc.cu -- diagnostics of a caller-held state without any device
// allocation.
//
// Some callers cannot allocate device memory at the point where they want the
// diagnostics: a host application whose memory pool already owns the free HBM
// (a cudaMalloc here would fail or compete with that pool), or a time-stepping
// loop that must not pay the device-wide synchronisation that cudaMalloc and
// cudaFree can cause.  For them, lbm_reduce_state_noalloc computes the same
// quantities as lbm_reduce from state arrays the caller already owns, using
// scratch space that lives in this file for the life of the process:
//
//   g_noalloc_scratch  kNoAllocMaxBlocks block partials + one result slot, each
//                      kDiagSlots doubles (about 786 KB).  Every GPU that loads
//                      the library holds one copy until the process exits.
//
// One block covers kNoAllocCellsPerBlock cells, so a box of at most
// kNoAllocMaxBlocks * kNoAllocCellsPerBlock = 134,217,728 cells (512^3) fits;
// larger boxes are rejected with LBM_ERR_ARG.  Every block overwrites its own
// partial and the final block overwrites the result slot, so nothing has to be
// cleared between calls; the array keeps the last call's contents.  All calls
// share the one array: calls whose work overlaps on the GPU (other streams,
// other host threads) race on it and must be serialised by the caller.
//
// Host code may not use the array's name as a device address: in host code it
// denotes a host-side stand-in.  The device address is obtained once per device
// with cudaGetSymbolAddress, with that device current, on the first call that
// runs on it, and kept for later calls (valid for the device's primary context:
// a cudaDeviceReset makes it stale, as the public header states).
#include <mutex>

#include "lbm_internal.h"

namespace lbm {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocCellsPerThread = 64;
constexpr int kNoAllocCellsPerBlock = kNoAllocThreads * kNoAllocCellsPerThread;  // 16384
constexpr int kNoAllocMaxBlocks = 8192;
constexpr long long kNoAllocMaxCells = (long long)kNoAllocMaxBlocks * kNoAllocCellsPerBlock;

static __device__ __align__(256) double g_noalloc_scratch[(kNoAllocMaxBlocks + 1) * kDiagSlots];

constexpr int kMaxDevices = 64;
static void *g_scratch_addr[kMaxDevices];
static std::mutex g_scratch_mutex;

// Device address of g_noalloc_scratch on the current device (set up once per device).
static cudaError_t scratch_address(int device, double **ptr) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[device] = p;
    }
    *ptr = static_cast<double *>(g_scratch_addr[device]);
    return cudaSuccess;
}

__device__ __forceinline__ double nwarp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double nwarp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Same per-cell quantities as the handle's reduction, read from g in the
// natural population layout; one partial per block of kNoAllocCellsPerBlock cells.
template <int QG>
__global__ void __launch_bounds__(kNoAllocThreads) noalloc_partial_kernel(Params p, const float *__restrict__ g,
                                                                          const float *__restrict__ phi,
                                                                          double *__restrict__ partials) {
    double acc[kDiagSlots];
#pragma unroll
    for (int k = 0; k < kDiagSlots; ++k) acc[k] = 0.0;
    const long long first = (long long)blockIdx.x * kNoAllocCellsPerBlock;
    for (int j = 0; j < kNoAllocCellsPerThread; ++j) {
        const long long c = first + (long long)j * kNoAllocThreads + threadIdx.x;
        if (c >= p.N) break;
        const int x = (int)(c % p.nx);
        const long long r = c / p.nx;
        const int y = (int)(r % p.ny);
        const int z = (int)(r / p.ny);
        const Cell C = make_cell(p, x, y, z);
        float nb[27];
        gather_phi(phi, C, nb);
        float gv[QG];
#pragma unroll
        for (int i = 0; i < QG; ++i) gv[i] = g[pop_src<QG, false>(C, p.N, i)];
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
        acc[11] = fmax(acc[11], sqrt((double)H.ux * H.ux + (double)H.uy * H.uy + (double)H.uz * H.uz));
    }
    __shared__ double sh[kNoAllocThreads / 32][kDiagSlots];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kDiagSlots; ++k) {
        const double v = (k == 11) ? nwarp_max(acc[k]) : nwarp_sum(acc[k]);
        if (lane == 0) sh[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < kDiagSlots) {
        const int k = threadIdx.x;
        double v = sh[0][k];
        for (int w = 1; w < kNoAllocThreads / 32; ++w) v = (k == 11) ? fmax(v, sh[w][k]) : v + sh[w][k];
        partials[(size_t)blockIdx.x * kDiagSlots + k] = v;
    }
}

__global__ void __launch_bounds__(kNoAllocThreads) noalloc_final_kernel(const double *__restrict__ partials,
                                                                        int nblocks, double *__restrict__ out) {
    __shared__ double sh[kNoAllocThreads / 32][kDiagSlots];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < kDiagSlots; ++k) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
            const double s = partials[(size_t)b * kDiagSlots + k];
            v = (k == 11) ? fmax(v, s) : v + s;
        }
        v = (k == 11) ? nwarp_max(v) : nwarp_sum(v);
        if (lane == 0) sh[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < kDiagSlots) {
        const int k = threadIdx.x;
        double v = sh[0][k];
        for (int w = 1; w < kNoAllocThreads / 32; ++w) v = (k == 11) ? fmax(v, sh[w][k]) : v + sh[w][k];
        out[k] = v;
    }
}

}  // namespace lbm

extern "C" {

lbm_status lbm_reduce_state_noalloc(const lbm_domain *dom, const lbm_params *prm, const float *g, const float *phi,
                                    double *out, void *cuda_stream) {
    using namespace lbm;
    if (!g || !phi || !out) return set_thread_error("null state or output pointer"), LBM_ERR_ARG;
    Params p;
    std::string why;
    const lbm_status st = prepare_problem(dom, prm, &p, &why);
    if (st != LBM_OK) return set_thread_error(why), st;
    if (p.N > kNoAllocMaxCells)
        return set_thread_error("lbm_reduce_state_noalloc handles at most 134217728 cells (512^3)"), LBM_ERR_ARG;
    int device = -1;
    cudaError_t e = cudaGetDevice(&device);
    double *scratch = nullptr;
    if (e == cudaSuccess) e = scratch_address(device, &scratch);
    if (e != cudaSuccess) return set_thread_error(std::string("scratch set-up: ") + cudaGetErrorString(e)), LBM_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int nblocks = (int)((p.N + kNoAllocCellsPerBlock - 1) / kNoAllocCellsPerBlock);
    double *result = scratch + (size_t)kNoAllocMaxBlocks * kDiagSlots;
    if (dom->q_hydro == 9)
        noalloc_partial_kernel<9><<<nblocks, kNoAllocThreads, 0, s>>>(p, g, phi, scratch);
    else if (dom->q_hydro == 19)
        noalloc_partial_kernel<19><<<nblocks, kNoAllocThreads, 0, s>>>(p, g, phi, scratch);
    else
        noalloc_partial_kernel<27><<<nblocks, kNoAllocThreads, 0, s>>>(p, g, phi, scratch);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        noalloc_final_kernel<<<1, kNoAllocThreads, 0, s>>>(scratch, nblocks, result);
        e = cudaGetLastError();
    }
    double raw[LBM_DIAG_COUNT];
    if (e == cudaSuccess) e = cudaMemcpyAsync(raw, result, sizeof(raw), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_thread_error(cudaGetErrorString(e)), LBM_ERR_CUDA;
    const double V = raw[LBM_DIAG_LIGHT_VOL];
    for (int k = 0; k < LBM_DIAG_COUNT; ++k) out[k] = raw[k];
    for (int k = LBM_DIAG_LIGHT_X; k <= LBM_DIAG_LIGHT_UZ; ++k) out[k] = V != 0.0 ? raw[k] / V : 0.0;
    return LBM_OK;
}

}  // extern "C"
