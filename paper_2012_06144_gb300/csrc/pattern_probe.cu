// pattern_probe.cu -- the DRAM bandwidth of the fused step's data movement
// without its arithmetic: a ceiling for the step's roofline fraction.
//
// The coupled update (Algorithm 2) reads and writes every population of both
// lattices once per cell and step (the byte count of Section 5.1).  How fast HBM serves
// that traffic depends on where the reads and writes fall: the AA pattern keeps one
// copy of each lattice and alternates a natural step (read and write at the cell)
// with a swapped step (read at x - e_i, write at x + e_i); in the fused kernel one
// lattice is natural while the other is swapped.  This program moves Q = 42 SoA
// planes of n^3 FP32 values (the D3Q15 + D3Q27 pair) with one thread per cell in
// the fused kernel's 32 x 2 x 4 blocks, with no arithmetic, under each pattern,
// and prints one JSON line of GB/s (bytes read + written / time, CUDA events over
// `iters` launches after 3 untimed ones):
//   copy     float4 copy of half the planes into the other half (a STREAM copy)
//   local    read and write every plane at the cell
//   aa_mix   21 planes local, 21 read at x - e and written at x + e (the fused step)
//   aa_odd   every plane read at x - e and written at x + e
//   pull     read at x - e, write at the cell (two grids)
//   push     read at the cell, write at x + e (two grids)
//   twist    read and write at x + max(e, 0) (the esoteric-twist locations)
// Plane s moves along direction s mod 27 of {-1, 0, 1}^3; periodic box, n a power
// of two and a multiple of 32.  Two buffers of 42 n^3 floats (45 GB at n = 512).
//
// Usage: pattern_probe [n=512] [iters=20]
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>

namespace {

constexpr int Q = 42, BX = 32, BY = 2, BZ = 4;

enum Pattern { LOCAL, AA_MIX, AA_ODD, PULL, PUSH, TWIST };

__device__ __forceinline__ int3 direction(int s) {
    const int d = s % 27;
    return make_int3(d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1);
}

// read shift r and write shift w of plane s (cells: read x + r, write x + w)
template <int P>
__device__ __forceinline__ void shifts(int s, int3 &r, int3 &w) {
    const int3 e = direction(s), z = make_int3(0, 0, 0);
    const int3 m = make_int3(-e.x, -e.y, -e.z);
    const int3 t = make_int3(max(e.x, 0), max(e.y, 0), max(e.z, 0));
    r = w = z;
    if (P == AA_MIX && s >= Q / 2) { r = m; w = e; }
    if (P == AA_ODD) { r = m; w = e; }
    if (P == PULL) r = m;
    if (P == PUSH) w = e;
    if (P == TWIST) r = w = t;
}

template <int P>
__global__ void __launch_bounds__(BX *BY *BZ, 4) move(const float *__restrict__ f, float *__restrict__ o, int n,
                                                      unsigned long long N) {
    const int nbx = n / BX, m = n - 1;
    const int by = blockIdx.x / nbx, bx = blockIdx.x - by * nbx;
    const int x = bx * BX + threadIdx.x, y = by * BY + threadIdx.y, z = blockIdx.y * BZ + threadIdx.z;
    float v[Q];
#pragma unroll
    for (int s = 0; s < Q; ++s) {
        int3 r, w;
        shifts<P>(s, r, w);
        const size_t c = (size_t)((x + r.x) & m) + (size_t)n * (((y + r.y) & m) + (size_t)n * ((z + r.z) & m));
        v[s] = __ldg(f + s * N + c);
    }
#pragma unroll
    for (int s = 0; s < Q; ++s) {
        int3 r, w;
        shifts<P>(s, r, w);
        const size_t c = (size_t)((x + w.x) & m) + (size_t)n * (((y + w.y) & m) + (size_t)n * ((z + w.z) & m));
        o[s * N + c] = v[s] * 1.0000001f;
    }
}

__global__ void copy4(const float4 *__restrict__ a, float4 *__restrict__ b, size_t n4) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x)
        b[i] = __ldg(a + i);
}

bool check(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return true;
    std::fprintf(stderr, "%s: %s\n", what, cudaGetErrorString(e));
    return false;
}

template <typename Launch>
double time_gbs(Launch launch, double bytes, int iters) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    for (int i = 0; i < 3; ++i) launch();
    cudaEventRecord(a);
    for (int i = 0; i < iters; ++i) launch();
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (cudaGetLastError() != cudaSuccess || ms <= 0.f) return -1.0;
    return bytes / (ms / iters / 1e3) / 1e9;
}

}  // namespace

int main(int argc, char **argv) {
    const int n = argc > 1 ? std::atoi(argv[1]) : 512;
    const int iters = argc > 2 ? std::atoi(argv[2]) : 20;
    if (n < 32 || n > 512 || (n & (n - 1)) != 0 || iters < 1) {
        std::fprintf(stderr, "n must be a power of two in [32, 512], iters >= 1\n");
        return 2;
    }
    const unsigned long long N = (unsigned long long)n * n * n;
    float *f = nullptr, *o = nullptr;
    if (!check(cudaMalloc(&f, Q * N * sizeof(float)), "cudaMalloc") ||
        !check(cudaMalloc(&o, Q * N * sizeof(float)), "cudaMalloc") ||
        !check(cudaMemset(f, 0, Q * N * sizeof(float)), "cudaMemset") ||
        !check(cudaMemset(o, 0, Q * N * sizeof(float)), "cudaMemset"))
        return 1;
    const dim3 grid((n / BX) * (n / BY), n / BZ), block(BX, BY, BZ);
    const double bytes = 2.0 * Q * N * sizeof(float);
    const size_t half4 = (size_t)(Q / 2) * N / 4;
    const double copy = time_gbs([&] { copy4<<<152 * 8, 512>>>((const float4 *)f, (float4 *)f + half4, half4); },
                                 2.0 * half4 * sizeof(float4), iters);
    const double local = time_gbs([&] { move<LOCAL><<<grid, block>>>(f, o, n, N); }, bytes, iters);
    const double aa_mix = time_gbs([&] { move<AA_MIX><<<grid, block>>>(f, o, n, N); }, bytes, iters);
    const double aa_odd = time_gbs([&] { move<AA_ODD><<<grid, block>>>(f, o, n, N); }, bytes, iters);
    const double pull = time_gbs([&] { move<PULL><<<grid, block>>>(f, o, n, N); }, bytes, iters);
    const double push = time_gbs([&] { move<PUSH><<<grid, block>>>(f, o, n, N); }, bytes, iters);
    const double twist = time_gbs([&] { move<TWIST><<<grid, block>>>(f, o, n, N); }, bytes, iters);
    const bool ok = check(cudaGetLastError(), "launch");
    cudaFree(f);
    cudaFree(o);
    if (!ok) return 1;
    std::printf("{\"n\": %d, \"planes\": %d, \"iters\": %d, \"unit\": \"GB/s\", \"copy\": %.1f, \"local\": %.1f, "
                "\"aa_mix\": %.1f, \"aa_odd\": %.1f, \"pull\": %.1f, \"push\": %.1f, \"twist\": %.1f}\n",
                n, Q, iters, copy, local, aa_mix, aa_odd, pull, push, twist);
    return 0;
}
