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
// of two and a multiple of 32.  Two buffers of 43 n^3 floats (46 GB at n = 512).
// Also, for n >= 64, the two-cell step's mix (move_pair below) in FP32 and with
// 16-bit moving populations:
//   pair32_g_natural / pair32_g_swapped   the FP32 step's accesses, per AA layout
//   pair16_g_natural / pair16_g_swapped   the same with 16-bit moving planes
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

// The two-cell step's data movement: a thread owns cells (x, x + 1), x even, in
// 64 x 2 x 2-cell blocks; the moving populations of D3Q27 (26 planes, g) and D3Q15
// (14 planes, h) in type T (float or 16-bit), two FP32 rest planes and an FP32 phi
// plane, 344 B (FP32) or 184 B (16-bit) per cell.  G_SW: g swapped and h natural,
// else g natural and h swapped.  A natural plane and a swapped plane with e_x = 0
// move one aligned pair per thread (at x - e read, x + e written); a swapped plane
// with e_x != 0 moves one element per cell, as the two-cell step does.
__device__ __forceinline__ int3 dir27(int i) {  // i in [0, 26): the nonzero vectors of {-1, 0, 1}^3
    const int d = i < 13 ? i : i + 1;
    return make_int3(d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1);
}
__device__ __forceinline__ int3 dir15(int i) {  // i in [0, 14): the six faces, then the eight corners
    if (i < 6) return make_int3(i / 2 == 0 ? 1 - 2 * (i & 1) : 0, i / 2 == 1 ? 1 - 2 * (i & 1) : 0,
                                i / 2 == 2 ? 1 - 2 * (i & 1) : 0);
    const int c = i - 6;
    return make_int3(c & 1 ? 1 : -1, c & 2 ? 1 : -1, c & 4 ? 1 : -1);
}

template <typename T>
struct Pair2 {
    using type = ushort2;
};
template <>
struct Pair2<float> {
    using type = float2;
};
template <typename T>
__device__ __forceinline__ T touch(T v) {
    if constexpr (sizeof(T) == 4) return v * 1.0000001f;
    else return (T)(v ^ 1u);
}

template <typename T, bool SW>
__device__ __forceinline__ void move_plane(const T *__restrict__ f, T *__restrict__ o, int3 e, int x, int y, int z,
                                           int n) {
    using P = typename Pair2<T>::type;
    const int m = n - 1;
    auto at = [&](int xx, int yy, int zz) {
        return (size_t)(xx & m) + (size_t)n * ((size_t)(yy & m) + (size_t)n * (size_t)(zz & m));
    };
    if (!SW || e.x == 0) {
        const int3 r = SW ? make_int3(-e.x, -e.y, -e.z) : make_int3(0, 0, 0);
        const int3 w = SW ? e : make_int3(0, 0, 0);
        P v = __ldg(reinterpret_cast<const P *>(f + at(x + r.x, y + r.y, z + r.z)));
        v.x = touch(v.x);
        v.y = touch(v.y);
        *reinterpret_cast<P *>(o + at(x + w.x, y + w.y, z + w.z)) = v;
        return;
    }
    const T a = __ldg(f + at(x - e.x, y - e.y, z - e.z)), b = __ldg(f + at(x + 1 - e.x, y - e.y, z - e.z));
    o[at(x + e.x, y + e.y, z + e.z)] = touch(a);
    o[at(x + 1 + e.x, y + e.y, z + e.z)] = touch(b);
}

template <typename T, bool G_SW>
__global__ void __launch_bounds__(128, 4) move_pair(const T *__restrict__ f, T *__restrict__ o,
                                                     const float *__restrict__ fr, float *__restrict__ orr, int n,
                                                     unsigned long long N) {
    const int nbx = n / 64;
    const int by = blockIdx.x / nbx, bx = blockIdx.x - by * nbx;
    const int x = bx * 64 + 2 * threadIdx.x, y = by * 2 + threadIdx.y, z = blockIdx.y * 2 + threadIdx.z;
    const size_t c = (size_t)x + (size_t)n * ((size_t)y + (size_t)n * z);
#pragma unroll
    for (int k = 0; k < 3; ++k) {  // the two rest planes and phi, at the cells
        float2 v = __ldg(reinterpret_cast<const float2 *>(fr + k * N + c));
        v.x *= 1.0000001f;
        v.y *= 1.0000001f;
        *reinterpret_cast<float2 *>(orr + k * N + c) = v;
    }
#pragma unroll
    for (int i = 0; i < 26; ++i) move_plane<T, G_SW>(f + i * N, o + i * N, dir27(i), x, y, z, n);
#pragma unroll
    for (int i = 0; i < 14; ++i) move_plane<T, !G_SW>(f + (26 + i) * N, o + (26 + i) * N, dir15(i), x, y, z, n);
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
    const unsigned long long planes = Q + 1;  // the two-cell mix moves 43 FP32 planes
    if (!check(cudaMalloc(&f, planes * N * sizeof(float)), "cudaMalloc") ||
        !check(cudaMalloc(&o, planes * N * sizeof(float)), "cudaMalloc") ||
        !check(cudaMemset(f, 0, planes * N * sizeof(float)), "cudaMemset") ||
        !check(cudaMemset(o, 0, planes * N * sizeof(float)), "cudaMemset"))
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
    // the two-cell step's mix: 40 moving planes (26 + 14) from the start of each
    // buffer, then the two rest planes and phi in FP32 after them (16-bit: the 40
    // planes fill 20 float planes); boxes of at least 64 cells along x
    double pair32[2] = {-1.0, -1.0}, pair16[2] = {-1.0, -1.0};
    if (n >= 64) {
        const dim3 pgrid((n / 64) * (n / 2), n / 2), pblock(32, 2, 2);
        auto *f16 = reinterpret_cast<unsigned short *>(f), *o16 = reinterpret_cast<unsigned short *>(o);
        pair32[0] = time_gbs([&] { move_pair<float, false><<<pgrid, pblock>>>(f, o, f + 40 * N, o + 40 * N, n, N); },
                             344.0 * N, iters);
        pair32[1] = time_gbs([&] { move_pair<float, true><<<pgrid, pblock>>>(f, o, f + 40 * N, o + 40 * N, n, N); },
                             344.0 * N, iters);
        pair16[0] = time_gbs(
            [&] { move_pair<unsigned short, false><<<pgrid, pblock>>>(f16, o16, f + 20 * N, o + 20 * N, n, N); },
            184.0 * N, iters);
        pair16[1] = time_gbs(
            [&] { move_pair<unsigned short, true><<<pgrid, pblock>>>(f16, o16, f + 20 * N, o + 20 * N, n, N); },
            184.0 * N, iters);
    }
    const bool ok = check(cudaGetLastError(), "launch");
    cudaFree(f);
    cudaFree(o);
    if (!ok) return 1;
    std::printf("{\"n\": %d, \"planes\": %d, \"iters\": %d, \"unit\": \"GB/s\", \"copy\": %.1f, \"local\": %.1f, "
                "\"aa_mix\": %.1f, \"aa_odd\": %.1f, \"pull\": %.1f, \"push\": %.1f, \"twist\": %.1f, "
                "\"pair32_g_natural\": %.1f, \"pair32_g_swapped\": %.1f, \"pair16_g_natural\": %.1f, "
                "\"pair16_g_swapped\": %.1f}\n",
                n, Q, iters, copy, local, aa_mix, aa_odd, pull, push, twist, pair32[0], pair32[1], pair16[0],
                pair16[1]);
    return 0;
}
