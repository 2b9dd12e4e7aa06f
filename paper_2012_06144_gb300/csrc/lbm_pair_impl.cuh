// lbm_pair_impl.cuh -- device code of the fused coupled step with two cells per
// thread, shared by the single-simulation kernel (lbm_pair.cu) and the batched
// kernel (lbm_batch.cu).
//
// The same update as fused_step_kernel (lbm_step.cu): one launch K_k advances
// every cell by the hydrodynamic step k-1 and the phase-field step k of
// Algorithm 2 (arXiv 2012.06144, Section 4.2), with the in-place AA streaming of
// both lattices.  Here a thread owns the two neighbouring cells (x, x + 1),
// x even, of one row, so that
//   * the arithmetic of the two cells runs as packed FP32 pairs (one f32x2
//     add, multiply or fused multiply-add of sm_100 and later per operation for
//     both cells), halving the arithmetic instructions of the step;
//   * a population whose two locations are neighbours in memory -- every
//     population of the lattice in natural layout, and those of the swapped
//     lattice that do not move along x -- is read and written as one 32-bit
//     (16-bit storage) or 64-bit (FP32) access for both cells; the others (the
//     swapped lattice's x-moving populations, whose locations x - e_x and
//     x + 1 - e_x straddle two aligned pairs or wrap around the box) take one
//     access per cell.
// Needs nx even (so that every pair starts on an even element and a thread's
// two cells are both inside or both outside the box); plane offsets in 32 bits
// ((q - 1) N < 2^32) or, for larger FP32 boxes, in 64 bits; the D3Q15 phase
// lattice with the SRT collision (or, in FP32, the MRT one) and D3Q19 or D3Q27
// hydrodynamics (and, in FP32, the other lattice pairs of Section 5.1).
//
// The arithmetic follows the single-cell kernel term by term (lbm_device.cuh,
// lbm_step_impl.cuh) with the same reformulations: stencils from opposite-pair
// differences grouped by weight class, moments from opposite-pair sums (D3Q27:
// the x-y-z cascade), rest populations as exact remainders of the zeroth
// moments, both lattices kept in their 16-bit storage units through the step.
// Rounding differs from the single-cell kernel only where a multiply and an add
// are fused differently.
#pragma once

#include "lbm_step_impl.cuh"

#ifndef LBM_PAIR_MIN_BLOCKS
#define LBM_PAIR_MIN_BLOCKS 4  // resident blocks per SM the register budget is sized for (128 registers)
#endif
#ifndef LBM_PAIR_MIXED
#define LBM_PAIR_MIXED 1  // 16-bit storage: sums of stored values by mixed-precision adds (0: convert, then add)
#endif

namespace lbm {
namespace pairstep {

constexpr int PX = 2 * TX;  // cells per block row: 32 threads x 2 cells
#ifndef LBM_PAIR_TY
#define LBM_PAIR_TY 2
#endif
#ifndef LBM_PAIR_TZ
#define LBM_PAIR_TZ 2
#endif
constexpr int TY = LBM_PAIR_TY, TZ = LBM_PAIR_TZ;  // block tile: 64 x TY x TZ cells
constexpr int ROW = PX + 4;  // phi tile row: columns 0..67 hold x0 - 2 .. x0 + 65

// ---- packed FP32 arithmetic on (cell x, cell x + 1)
__device__ __forceinline__ float2 bc(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 mul(float2 a, float s) { return __fmul2_rn(a, bc(s)); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fma2(float2 a, float s, float2 c) { return __ffma2_rn(a, bc(s), c); }
// a - b, exactly rounded: fma(b, -1, a)
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return __ffma2_rn(b, bc(-1.0f), a); }
// acc + d or acc - d for a direction component of sign s (compile time)
__device__ __forceinline__ float2 acc_signed(float2 acc, float2 d, int s) { return s > 0 ? add(acc, d) : sub(acc, d); }

// ---- storage pairs: two consecutive elements of a plane
template <typename T>
struct PairOf;
template <>
struct PairOf<float> {
    using P = float2;
};
template <>
struct PairOf<__half> {
    using P = __half2;
};
template <>
struct PairOf<__nv_bfloat16> {
    using P = __nv_bfloat162;
};

template <typename T>
__device__ __forceinline__ float2 unpack(typename PairOf<T>::P v) {
    if constexpr (std::is_same<T, __half>::value) return __half22float2(v);
    else if constexpr (std::is_same<T, __nv_bfloat16>::value) return __bfloat1622float2(v);
    else return v;
}

template <typename T>
__device__ __forceinline__ typename PairOf<T>::P pack(float2 v) {
    if constexpr (std::is_same<T, __half>::value) return __float22half2_rn(v);
    else if constexpr (std::is_same<T, __nv_bfloat16>::value) return __float22bfloat162_rn(v);
    else return v;
}

template <typename T>
__device__ __forceinline__ T lo(typename PairOf<T>::P v) {
    if constexpr (std::is_same<T, __half>::value) return __low2half(v);
    else if constexpr (std::is_same<T, __nv_bfloat16>::value) return __low2bfloat16(v);
    else return v.x;
}

template <typename T>
__device__ __forceinline__ T hi(typename PairOf<T>::P v) {
    if constexpr (std::is_same<T, __half>::value) return __high2half(v);
    else if constexpr (std::is_same<T, __nv_bfloat16>::value) return __high2bfloat16(v);
    else return v.y;
}

template <typename T>
__device__ __forceinline__ typename PairOf<T>::P join(T a, T b) {
    if constexpr (std::is_same<T, __half>::value) return __halves2half2(a, b);
    else if constexpr (std::is_same<T, __nv_bfloat16>::value) return __halves2bfloat162(a, b);
    else return make_float2(a, b);
}

// Mixed-precision add and subtract of sm_100 and later: the 16-bit operand is
// widened inside the FP32 operation (cvt(a) + c, cvt(a) - c), which spares the
// separate conversion -- on this GPU a conversion costs the multiply-add pipe
// twice what an add does, and the 16-bit steps are held back by that pipe.
template <typename T>
__device__ __forceinline__ float madd(T a, float c) {
    float d;
    if constexpr (std::is_same<T, __half>::value)
        asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(__half_as_ushort(a)), "f"(c));
    else
        asm("add.rn.f32.bf16 %0, %1, %2;" : "=f"(d) : "h"(__bfloat16_as_ushort(a)), "f"(c));
    return d;
}

template <typename T>
__device__ __forceinline__ float msub(T a, float c) {
    float d;
    if constexpr (std::is_same<T, __half>::value)
        asm("sub.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(__half_as_ushort(a)), "f"(c));
    else
        asm("sub.rn.f32.bf16 %0, %1, %2;" : "=f"(d) : "h"(__bfloat16_as_ushort(a)), "f"(c));
    return d;
}

// the same for both cells of a stored pair: cvt(q) + c, cvt(q) - c
template <typename T>
__device__ __forceinline__ float2 madd2(typename PairOf<T>::P q, float2 c) {
    return make_float2(madd<T>(lo<T>(q), c.x), madd<T>(hi<T>(q), c.y));
}
template <typename T>
__device__ __forceinline__ float2 msub2(typename PairOf<T>::P q, float2 c) {
    return make_float2(msub<T>(lo<T>(q), c.x), msub<T>(hi<T>(q), c.y));
}

// One lattice: FP32 rest plane and q - 1 moving planes of type T, element offsets
// (s - 1) N + idx in 32 bits, or (W64) in 64 bits for boxes with (q - 1) N >= 2^32.
template <typename T, bool W64 = false>
struct Lat {
    float *rest;
    T *mov;
    unsigned N;
    __device__ __forceinline__ T *at(int s, int idx) const {
        if constexpr (W64) return mov + ((size_t)(s - 1) * N + (size_t)(unsigned)idx);
        else return mov + ((unsigned)(s - 1) * N + (unsigned)idx);
    }
};

// Per-thread offsets of the pair: X[k] is the element index of x - 1 + k in the
// cells' row (k = 0..3; periodic wrap, or clamp at a walled face), Y / Z the
// offsets of the neighbouring rows / planes (0 at the centre); lo / hi the walled
// faces touched by cell A = x (bits of lo[0], hi[0]) and cell B = x + 1.
struct Nb4 {
    int X[4], Y[3], Z[3];
    int lo[2], hi[2];
};

__device__ __forceinline__ int nidx(const Nb4 &n, int k, int dx, int dy, int dz) {
    return n.X[1 + k + dx] + n.Y[dy + 1] + n.Z[dz + 1];
}

// True if cell k's x + sign e leaves the box through a wall (EDGE: 0 no walls in
// the tile, 1 the x walls only, 7 any).
template <int EDGE>
__device__ __forceinline__ bool leaves(const Nb4 &n, int k, V3 e, int sign) {
    if constexpr (EDGE == 0) return false;
    const int ex = e.x * sign, ey = e.y * sign, ez = e.z * sign;
    if constexpr (EDGE == 1) return (ex > 0 && (n.hi[k] & 1)) || (ex < 0 && (n.lo[k] & 1));
    return (ex > 0 && (n.hi[k] & 1)) || (ex < 0 && (n.lo[k] & 1)) || (ey > 0 && (n.hi[k] & 2)) ||
           (ey < 0 && (n.lo[k] & 2)) || (ez > 0 && (n.hi[k] & 4)) || (ez < 0 && (n.lo[k] & 4));
}

// (slot, element) of the pre-collision f_i of cell k (AA layout, lbm_device.cuh)
template <int Q, bool SW, int EDGE>
__device__ __forceinline__ void src(const Nb4 &n, int k, int i, int &slot, int &idx) {
    const V3 e = vel<Q>(i);
    if (!SW || leaves<EDGE>(n, k, e, -1)) {
        slot = i;
        idx = n.X[1 + k];
        return;
    }
    slot = opp(i);
    idx = nidx(n, k, -e.x, -e.y, -e.z);
}

// (slot, element) receiving the post-collision f*_i of cell k
template <int Q, bool SW, int EDGE>
__device__ __forceinline__ void dst(const Nb4 &n, int k, int i, int &slot, int &idx) {
    const V3 e = vel<Q>(i);
    if (!SW || leaves<EDGE>(n, k, e, +1)) {
        slot = opp(i);
        idx = n.X[1 + k];
        return;
    }
    slot = i;
    idx = nidx(n, k, e.x, e.y, e.z);
}

// True if both cells' locations of population i form one aligned pair: always in
// natural layout; in swapped layout when e_x = 0 (y and z bounce-back is the
// same for both cells of a row).
template <int Q, bool SW>
__device__ __forceinline__ constexpr bool paired(int i) {
    return !SW || vel<Q>(i).x == 0;
}

// Pre-collision moving population f_i (i > 0) of both cells as stored (a
// packed pair of the storage type; converted where it is used, so that the
// loaded state occupies one register per population pair in 16-bit storage).
template <typename T, int Q, bool SW, int EDGE, bool W64 = false>
__device__ __forceinline__ typename PairOf<T>::P load_pop(const Lat<T, W64> &L, const Nb4 &n, int i) {
    using P = typename PairOf<T>::P;
    if (paired<Q, SW>(i)) {
        int slot, idx;
        src<Q, SW, EDGE>(n, 0, i, slot, idx);
        return ld_pop(reinterpret_cast<const P *>(L.at(slot, idx)));
    }
    int sa, ia, sb, ib;
    src<Q, SW, EDGE>(n, 0, i, sa, ia);
    src<Q, SW, EDGE>(n, 1, i, sb, ib);
    return join<T>(ld_pop(L.at(sa, ia)), ld_pop(L.at(sb, ib)));
}

// the rest population of both cells (FP32, always at the cells themselves)
__device__ __forceinline__ float2 load_rest(const float *rest, const Nb4 &n) {
    return ld_pop(reinterpret_cast<const float2 *>(rest + n.X[1]));
}

// Stores the encoded post-collision f*_i of both cells.
template <typename T, int Q, bool SW, int EDGE, bool W64 = false>
__device__ __forceinline__ void store_pop(const Lat<T, W64> &L, const Nb4 &n, int i, typename PairOf<T>::P v) {
    using P = typename PairOf<T>::P;
    if (paired<Q, SW>(i)) {
        int slot, idx;
        dst<Q, SW, EDGE>(n, 0, i, slot, idx);
        *reinterpret_cast<P *>(L.at(slot, idx)) = v;
        return;
    }
    int sa, ia, sb, ib;
    dst<Q, SW, EDGE>(n, 0, i, sa, ia);
    dst<Q, SW, EDGE>(n, 1, i, sb, ib);
    st_pop(L.at(sa, ia), lo<T>(v));
    st_pop(L.at(sb, ib), hi<T>(v));
}

// the rest population (always at the cells themselves)
__device__ __forceinline__ void store_rest(float *rest, const Nb4 &n, float2 v) {
    *reinterpret_cast<float2 *>(rest + n.X[1]) = v;
}

// Class sums of eq:grad / eq:lap for both cells (see stencil_sums), read from the
// phi tile row by row: each row of the 3 x 3 neighbourhood is met together with
// its opposite row, so only two rows are live at a time.
struct Stencil2 {
    float2 D1[3], D2[3], D3[3];
    float2 L1, L2, L3;
};

struct Row3 {
    float2 L, M, R;  // (x - 1, x), (x, x + 1), (x + 1, x + 2) of the row
    __device__ __forceinline__ float2 at(int ex) const { return ex < 0 ? L : (ex > 0 ? R : M); }
};

// a tile row from the thread's columns: (x - 2, x - 1), (x, x + 1), (x + 2, x + 3)
__device__ __forceinline__ Row3 tile_row(const float *row) {
    const float2 a = *reinterpret_cast<const float2 *>(row), m = *reinterpret_cast<const float2 *>(row + 2),
                 r = *reinterpret_cast<const float2 *>(row + 4);
    return Row3{make_float2(a.y, m.x), m, make_float2(m.y, r.x)};
}

// the opposite pair (e, -e) with phi(x + e) = vp, phi(x - e) = vm into the class sums
__device__ __forceinline__ void stencil_pair(Stencil2 &S, float2 vp, float2 vm, float2 c, int ex, int ey, int ez) {
    const float2 D = sub(vp, vm), L = add(sub(vp, c), sub(vm, c));
    const int cls = ex * ex + ey * ey + ez * ez;
    float2 *Dc = cls == 1 ? S.D1 : (cls == 2 ? S.D2 : S.D3);
    if (ex) Dc[0] = acc_signed(Dc[0], D, ex);
    if (ey) Dc[1] = acc_signed(Dc[1], D, ey);
    if (ez) Dc[2] = acc_signed(Dc[2], D, ez);
    if (cls == 1) S.L1 = add(S.L1, L);
    else if (cls == 2) S.L2 = add(S.L2, L);
    else S.L3 = add(S.L3, L);
}

// rows(dy, dz): pointer to the tile row at offset (dy, dz) from the cells' row at
// the thread's columns; centre receives phi of both cells
// PLANE: the in-plane neighbours only (the D2Q9 pair on an nx x ny x 1 box).
template <bool PLANE = false, typename RowPtr>
__device__ __forceinline__ Stencil2 stencil_from_tile(const RowPtr &rows, float2 &centre) {
    Stencil2 S;
#pragma unroll
    for (int a = 0; a < 3; ++a) S.D1[a] = S.D2[a] = S.D3[a] = bc(0.f);
    S.L1 = S.L2 = S.L3 = bc(0.f);
    const Row3 r0 = tile_row(rows(0, 0));
    const float2 c = r0.M;
    centre = c;
    stencil_pair(S, r0.R, r0.L, c, 1, 0, 0);
    constexpr int DY[4] = {1, 0, 1, 1}, DZ[4] = {0, 1, 1, -1};
#pragma unroll
    for (int k = 0; k < (PLANE ? 1 : 4); ++k) {
        const Row3 rp = tile_row(rows(DY[k], DZ[k])), rm = tile_row(rows(-DY[k], -DZ[k]));
#pragma unroll
        for (int ex = -1; ex <= 1; ++ex) stencil_pair(S, rp.at(ex), rm.at(-ex), c, ex, DY[k], DZ[k]);
    }
    return S;
}

template <int Q>
__device__ __forceinline__ void grad2(const Stencil2 &S, float2 &gx, float2 &gy, float2 &gz) {
    constexpr float w1 = 3.f * wclass<Q>(1), w2 = 3.f * wclass<Q>(2), w3 = 3.f * wclass<Q>(3);
    float2 g[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        g[a] = mul(S.D1[a], w1);
        if (w2 != 0.f) g[a] = fma2(S.D2[a], w2, g[a]);
        if (w3 != 0.f) g[a] = fma2(S.D3[a], w3, g[a]);
    }
    gx = g[0];
    gy = g[1];
    gz = g[2];
}

template <int Q>
__device__ __forceinline__ float2 lap2(const Stencil2 &S) {
    constexpr float w1 = 6.f * wclass<Q>(1), w2 = 6.f * wclass<Q>(2), w3 = 6.f * wclass<Q>(3);
    float2 l = mul(S.L1, w1);
    if (w2 != 0.f) l = fma2(S.L2, w2, l);
    if (w3 != 0.f) l = fma2(S.L3, w3, l);
    return l;
}

// moments of g (storage units) up to second order: p*, j, the second moments
struct Moments2 {
    float2 ps, jx, jy, jz, mxx, myy, mzz, mxy, mxz, myz;
};

template <int QG, typename G>
__device__ __forceinline__ Moments2 moments2(const G &gv) {
    Moments2 M;
    if constexpr (QG == 27) {
        // the x-y-z cascade of hydro_macro
        float2 X0[3][3], X1[3][3], X2[3][3];
#pragma unroll
        for (int z = 0; z < 3; ++z)
#pragma unroll
            for (int y = 0; y < 3; ++y) {
                const float2 a = gv(idx27(-1, y - 1, z - 1)), b = gv(idx27(0, y - 1, z - 1)),
                             c = gv(idx27(1, y - 1, z - 1));
                X2[z][y] = add(a, c);
                X0[z][y] = add(X2[z][y], b);
                X1[z][y] = sub(c, a);
            }
        float2 Y00[3], Y01[3], Y02[3], Y10[3], Y11[3], Y20[3];
#pragma unroll
        for (int z = 0; z < 3; ++z) {
            Y02[z] = add(X0[z][0], X0[z][2]);
            Y00[z] = add(Y02[z], X0[z][1]);
            Y01[z] = sub(X0[z][2], X0[z][0]);
            Y10[z] = add(add(X1[z][0], X1[z][2]), X1[z][1]);
            Y11[z] = sub(X1[z][2], X1[z][0]);
            Y20[z] = add(add(X2[z][0], X2[z][2]), X2[z][1]);
        }
        M.mzz = add(Y00[0], Y00[2]);
        M.ps = add(M.mzz, Y00[1]);
        M.jz = sub(Y00[2], Y00[0]);
        M.jy = add(add(Y01[0], Y01[2]), Y01[1]);
        M.myz = sub(Y01[2], Y01[0]);
        M.myy = add(add(Y02[0], Y02[2]), Y02[1]);
        M.jx = add(add(Y10[0], Y10[2]), Y10[1]);
        M.mxz = sub(Y10[2], Y10[0]);
        M.mxy = add(add(Y11[0], Y11[2]), Y11[1]);
        M.mxx = add(add(Y20[0], Y20[2]), Y20[1]);
    } else {
        M.ps = gv(0);
        M.jx = M.jy = M.jz = M.mxx = M.myy = M.mzz = M.mxy = M.mxz = M.myz = bc(0.f);
#pragma unroll
        for (int i = 1; i < QG; i += 2) {
            const V3 e = vel<QG>(i);
            const float2 s = add(gv(i), gv(i + 1)), d = sub(gv(i), gv(i + 1));
            M.ps = add(M.ps, s);
            if (e.x) { M.jx = acc_signed(M.jx, d, e.x); M.mxx = add(M.mxx, s); }
            if (e.y) { M.jy = acc_signed(M.jy, d, e.y); M.myy = add(M.myy, s); }
            if (e.z) { M.jz = acc_signed(M.jz, d, e.z); M.mzz = add(M.mzz, s); }
            if (e.x && e.y) M.mxy = acc_signed(M.mxy, s, e.x * e.y);
            if (e.x && e.z) M.mxz = acc_signed(M.mxz, s, e.x * e.z);
            if (e.y && e.z) M.myz = acc_signed(M.myz, s, e.y * e.z);
        }
    }
    return M;
}

// Pairwise sum a[LO] + ... + a[LO + N - 1], halves first (as tree_sum).
template <int LO, int N>
__device__ __forceinline__ float2 tree_sum2(const float2 *a) {
    if constexpr (N == 1) return a[LO];
    else return add(tree_sum2<LO, N / 2>(a), tree_sum2<LO + N / 2, N - N / 2>(a));
}

// The D3Q27 moments of 16-bit stored populations by the same x-y-z cascade, with
// each line's first-level sums taken by mixed-precision operations: per line
// (a, b, c) along x only a is converted; a + c, (a + c) + b and c - a widen c and
// b inside the adds.  The same sums, in the same order, as moments2.
template <typename T>
__device__ __forceinline__ Moments2 moments27_mixed(const typename PairOf<T>::P *gq, float2 g0) {
    float2 X0[3][3], X1[3][3], X2[3][3];
#pragma unroll
    for (int z = 0; z < 3; ++z)
#pragma unroll
        for (int y = 0; y < 3; ++y) {
            const int ia = idx27(-1, y - 1, z - 1), ib = idx27(0, y - 1, z - 1), ic = idx27(1, y - 1, z - 1);
            const float2 a = unpack<T>(gq[ia]);
            X2[z][y] = madd2<T>(gq[ic], a);
            X0[z][y] = ib == 0 ? add(X2[z][y], g0) : madd2<T>(gq[ib], X2[z][y]);
            X1[z][y] = msub2<T>(gq[ic], a);
        }
    Moments2 M;
    float2 Y00[3], Y01[3], Y02[3], Y10[3], Y11[3], Y20[3];
#pragma unroll
    for (int z = 0; z < 3; ++z) {
        Y02[z] = add(X0[z][0], X0[z][2]);
        Y00[z] = add(Y02[z], X0[z][1]);
        Y01[z] = sub(X0[z][2], X0[z][0]);
        Y10[z] = add(add(X1[z][0], X1[z][2]), X1[z][1]);
        Y11[z] = sub(X1[z][2], X1[z][0]);
        Y20[z] = add(add(X2[z][0], X2[z][2]), X2[z][1]);
    }
    M.mzz = add(Y00[0], Y00[2]);
    M.ps = add(M.mzz, Y00[1]);
    M.jz = sub(Y00[2], Y00[0]);
    M.jy = add(add(Y01[0], Y01[2]), Y01[1]);
    M.myz = sub(Y01[2], Y01[0]);
    M.myy = add(add(Y02[0], Y02[2]), Y02[1]);
    M.jx = add(add(Y10[0], Y10[2]), Y10[1]);
    M.mxz = sub(Y10[2], Y10[0]);
    M.mxy = add(add(Y11[0], Y11[2]), Y11[1]);
    M.mxx = add(add(Y20[0], Y20[2]), Y20[1]);
    return M;
}

// per-cell reciprocal (correctly rounded, as in the single-cell kernel)
__device__ __forceinline__ float2 rcp2(float2 v) { return make_float2(__frcp_rn(v.x), __frcp_rn(v.y)); }
__device__ __forceinline__ float2 clamp2(float2 v, float a, float b) {
    return make_float2(fminf(fmaxf(v.x, a), b), fminf(fmaxf(v.y, a), b));
}
__device__ __forceinline__ bool finite_pair(float2 v) { return fabsf(v.x) < 1e30f && fabsf(v.y) < 1e30f; }

// The collision of both lattices at the pair and the streaming stores, from the
// pre-collision populations gv (g^{k-1}, storage units), hv (h^k, storage units)
// and the neighbourhood nb of phi^{k-1}.  See collide_and_store.
// PMRT: the MRT phase collision of Section 3.1 (first-order moments relaxed with
// omega_phi, all others with 1) in the closed form of the one-cell kernel:
// h*_i = h^eq_i + F_i / 2 + 3 (1 - omega_phi) w_i e_i . J with
// J = sum_j e_j h_j - phi_k u + theta n / 6 (FP32 storage).
template <typename T, int QG, int QP, bool G_SW, bool H_SW, int EDGE, bool PMRT = false, bool W64 = false>
__device__ __forceinline__ void collide2(const Params &p, const Lat<T, W64> &lh, const Lat<T, W64> &lg, const Nb4 &n,
                                         float2 grest, const typename PairOf<T>::P *gq, float2 hrest,
                                         const typename PairOf<T>::P *hq, const Stencil2 &S, float2 phic,
                                         float *__restrict__ phi_out, int *__restrict__ flag) {
    using P = typename PairOf<T>::P;
    constexpr bool F32 = std::is_same<T, float>::value;

    // ---- hydrodynamic step k-1 (Section 3.2); g in storage units (the FP32 rest
    // population times the scale)
    const float2 g0 = F32 ? grest : mul(grest, p.g_scale);
    auto gv = [&](int i) { return i == 0 ? g0 : unpack<T>(gq[i]); };
    Moments2 M;
    if constexpr (!F32 && QG == 27 && LBM_PAIR_MIXED) M = moments27_mixed<T>(gq, g0);
    else M = moments2<QG>(gv);
    if constexpr (!F32) {  // storage units -> values (a power of two: exact)
        const float r = p.g_inv_scale;
        M.ps = mul(M.ps, r);
        M.jx = mul(M.jx, r);
        M.jy = mul(M.jy, r);
        M.jz = mul(M.jz, r);
        M.mxx = mul(M.mxx, r);
        M.myy = mul(M.myy, r);
        M.mzz = mul(M.mzz, r);
        M.mxy = mul(M.mxy, r);
        M.mxz = mul(M.mxz, r);
        M.myz = mul(M.myz, r);
    }
    float2 gpx, gpy, gpz;
    grad2<QG>(S, gpx, gpy, gpz);
    const float2 lap = lap2<QG>(S);
    const float2 phim = clamp2(phic, p.phi_lo, p.phi_hi);
    const float2 rho = fma2(phim, p.drho, bc(p.rho_L));  // eq:density
    const float2 hir = mul(rcp2(rho), 0.5f);
    const float2 tau = fma2(phim, p.dtau, bc(p.tau_L));
    const float2 s_nu = rcp2(add(tau, bc(0.5f)));
    const float2 grx = mul(gpx, p.drho), gry = mul(gpy, p.drho), grz = mul(gpz, p.drho);
    // eq:chemPot, eq:surfaceTension: mu = 4 beta phi (phi - 1)(phi - 1/2) - kappa lap
    const float2 cub = mul(mul(mul(phic, p.beta4), sub(phic, bc(1.0f))), sub(phic, bc(0.5f)));
    const float2 mu = fma2(lap, -p.kappa, cub);
    // eq:pressure_force, buoyancy
    const float2 cp = mul(M.ps, -1.0f / 3.0f);
    const float2 db = sub(rho, bc(p.rho_ref));
    const float2 f0x = fma2(db, p.gx, fma2(cp, grx, mul(mu, gpx)));
    const float2 f0y = fma2(db, p.gy, fma2(cp, gry, mul(mu, gpy)));
    const float2 f0z = fma2(db, p.gz, fma2(cp, grz, mul(mu, gpz)));
    // non-equilibrium second moments with u' (all forces but F_mu)
    const float2 upx = fma2(f0x, hir, M.jx), upy = fma2(f0y, hir, M.jy), upz = fma2(f0z, hir, M.jz);
    const float2 c3 = mul(M.ps, 1.0f / 3.0f);
    // Hermite second moments over the lattice's own dimensions (no zz for D2Q9)
    const float2 a2xx = sub(M.mxx, c3), a2yy = sub(M.myy, c3), a2zz = QG == 9 ? bc(0.f) : sub(M.mzz, c3);
    const float2 nupx = mul(upx, -1.0f), nupy = mul(upy, -1.0f), nupz = mul(upz, -1.0f);
    const float2 pxx = fma2(upx, nupx, a2xx), pyy = fma2(upy, nupy, a2yy), pzz = fma2(upz, nupz, a2zz);
    const float2 pxy = fma2(upx, nupy, M.mxy), pxz = fma2(upx, nupz, M.mxz), pyz = fma2(upy, nupz, M.myz);
    // eq:viscousForce: F_mu = -tau s_nu Pi_neq . grad rho
    const float2 cm = mul(mul(tau, s_nu), -1.0f);
    const float2 Fx = fma2(cm, fma2(pxz, grz, fma2(pxy, gry, mul(pxx, grx))), f0x);
    const float2 Fy = fma2(cm, fma2(pyz, grz, fma2(pyy, gry, mul(pxy, grx))), f0y);
    const float2 Fz = fma2(cm, fma2(pzz, grz, fma2(pyz, gry, mul(pxz, grx))), f0z);
    const float2 ux = fma2(Fx, hir, M.jx), uy = fma2(Fy, hir, M.jy), uz = fma2(Fz, hir, M.jz);

    // eq:improved_collision in Hermite form (hydro_post), coefficients scaled to
    // storage units
    {
        const float s = F32 ? 1.0f : p.g_scale;
        const float2 r = sub(bc(1.0f), s_nu);
        const float2 m0 = mul(M.ps, s);
        const float2 m1x = mul(fma2(Fx, hir, ux), 3.0f * s), m1y = mul(fma2(Fy, hir, uy), 3.0f * s),
                     m1z = mul(fma2(Fz, hir, uz), 3.0f * s);
        const float2 bxx = fma2(mul(s_nu, ux), ux, mul(r, a2xx));
        const float2 byy = fma2(mul(s_nu, uy), uy, mul(r, a2yy));
        const float2 bzz = fma2(mul(s_nu, uz), uz, mul(r, a2zz));
        const float2 Bxx = mul(bxx, 4.5f * s), Byy = mul(byy, 4.5f * s), Bzz = mul(bzz, 4.5f * s);
        const float2 Bxy = mul(fma2(mul(s_nu, ux), uy, mul(r, M.mxy)), 9.0f * s);
        const float2 Bxz = mul(fma2(mul(s_nu, ux), uz, mul(r, M.mxz)), 9.0f * s);
        const float2 Byz = mul(fma2(mul(s_nu, uy), uz, mul(r, M.myz)), 9.0f * s);
        const float2 m0t = sub(m0, mul(add(add(bxx, byy), bzz), 1.5f * s));
        // the rest population takes p* - sum_{i>0} g*_i over the stored values
        float2 gsum = bc(0.f);
#pragma unroll
        for (int i = 1; i < QG; i += 2) {
            const V3 e = vel<QG>(i);
            float2 ev = m0t, od = bc(0.f);
            if (e.x) { od = acc_signed(od, m1x, e.x); ev = add(ev, Bxx); }
            if (e.y) { od = acc_signed(od, m1y, e.y); ev = add(ev, Byy); }
            if (e.z) { od = acc_signed(od, m1z, e.z); ev = add(ev, Bzz); }
            if (e.x && e.y) ev = acc_signed(ev, Bxy, e.x * e.y);
            if (e.x && e.z) ev = acc_signed(ev, Bxz, e.x * e.z);
            if (e.y && e.z) ev = acc_signed(ev, Byz, e.y * e.z);
            const float w = wgt<QG>(i);
            const float2 E = mul(ev, w), O = mul(od, w);
            const P qa = pack<T>(add(E, O)), qb = pack<T>(sub(E, O));
            store_pop<T, QG, G_SW, EDGE>(lg, n, i, qa);
            store_pop<T, QG, G_SW, EDGE>(lg, n, i + 1, qb);
            if constexpr (!F32 && LBM_PAIR_MIXED) gsum = madd2<T>(qb, madd2<T>(qa, gsum));
            else gsum = add(gsum, add(unpack<T>(qa), unpack<T>(qb)));
        }
        if constexpr (!F32) gsum = mul(gsum, p.g_inv_scale);
        store_rest(lg.rest, n, sub(M.ps, gsum));
    }
    if (!finite_pair(M.ps)) *flag = 1;

    // ---- phase-field step k (Section 3.1), h in storage units q_i = h_i - w_i phi_ref
    const float href = F32 ? 0.0f : p.h_ref;
    float2 hv[QP];
    hv[0] = hrest;
#pragma unroll
    for (int i = 1; i < QP; ++i) hv[i] = unpack<T>(hq[i]);
    // phi_k = sum_i h_i (eq:updatePhaseField), as a tree over opposite pairs
    constexpr int NPR = (QP + 1) / 2;
    float2 pr[NPR];
    pr[0] = F32 ? hv[0] : add(hv[0], bc(href * (1.0f - wgt<QP>(0))));
#pragma unroll
    for (int j = 0; j < NPR - 1; ++j) pr[j + 1] = add(hv[2 * j + 1], hv[2 * j + 2]);
    const float2 phik = tree_sum2<0, NPR>(pr);
    *reinterpret_cast<float2 *>(phi_out + n.X[1]) = phik;
    if (!finite_pair(phik)) *flag = 1;

    float2 Gx, Gy, Gz;
    grad2<QP>(S, Gx, Gy, Gz);
    const float2 G2 = fma2(Gz, Gz, fma2(Gy, Gy, mul(Gx, Gx)));
    float2 inv = bc(0.f);
    if (G2.x > 1e-24f) inv.x = rsqrtf(G2.x);
    if (G2.y > 1e-24f) inv.y = rsqrtf(G2.y);
    // one Newton step: inv (1.5 - 0.5 G2 inv^2)
    inv = mul(inv, fma2(mul(G2, -0.5f), mul(inv, inv), bc(1.5f)));
    const float2 nx = mul(Gx, inv), ny = mul(Gy, inv), nz = mul(Gz, inv);
    const float2 pc = sub(phic, bc(0.5f));
    const float2 theta = mul(fma2(mul(pc, -4.0f), pc, bc(1.0f)), p.inv_xi);
    // -1.5 u.u
    const float2 nuu = mul(fma2(uz, uz, fma2(uy, uy, mul(ux, ux))), -1.5f);
    float om = p.omega_phi, fc = 1.0f - 0.5f * om;
    float2 cJx = bc(0.f), cJy = bc(0.f), cJz = bc(0.f);
    if constexpr (PMRT) {
        static_assert(F32, "the MRT phase collision is built for FP32 storage");
        float2 jx = bc(0.f), jy = bc(0.f), jz = bc(0.f);
#pragma unroll
        for (int i = 1; i < QP; i += 2) {
            const V3 e = vel<QP>(i);
            const float2 dh = sub(hv[i], hv[i + 1]);
            if (e.x) jx = acc_signed(jx, dh, e.x);
            if (e.y) jy = acc_signed(jy, dh, e.y);
            if (e.z) jz = acc_signed(jz, dh, e.z);
        }
        const float c = 3.0f * (1.0f - om);
        const float2 th = mul(theta, 0.5f / 3.0f);
        cJx = mul(sub(fma2(th, nx, jx), mul(phik, ux)), c);
        cJy = mul(sub(fma2(th, ny, jy), mul(phik, uy)), c);
        cJz = mul(sub(fma2(th, nz, jz), mul(phik, uz)), c);
        om = 1.0f;
        fc = 0.5f;
    }
    const float2 phin = F32 ? phik : sub(phik, bc(href));
    const float2 fth = mul(theta, fc);
    // per weight class c (|e|^2 = 1, 2, 3; the classes of the phase lattice):
    // phi_k w_c times 4.5, -1.5 u.u and 3 (the velocity terms of h^eq), and the
    // forcing factor (1 - omega/2) theta w_c
    float2 A[4], B[4], Tc[4], Fw[4];
#pragma unroll
    for (int c = 1; c <= 3; ++c) {
        const float wc = wclass<QP>(c);
        const float2 pwc = mul(phik, wc);
        A[c] = mul(pwc, 4.5f);
        B[c] = mul(pwc, nuu);
        Tc[c] = mul(pwc, 3.0f);
        Fw[c] = mul(fth, wc);
    }
    float2 dsum = bc(0.f);
#pragma unroll
    for (int i = 1; i < QP; i += 2) {
        const V3 e = vel<QP>(i);
        const float w = wgt<QP>(i);
        const int c = e.x * e.x + e.y * e.y + e.z * e.z;
        float2 eu = bc(0.f), en = bc(0.f);
        if (e.x) { eu = acc_signed(eu, ux, e.x); en = acc_signed(en, nx, e.x); }
        if (e.y) { eu = acc_signed(eu, uy, e.y); en = acc_signed(en, ny, e.y); }
        if (e.z) { eu = acc_signed(eu, uz, e.z); en = acc_signed(en, nz, e.z); }
        // velocity terms of h^eq: phi_k w (4.5 (e.u)^2 - 1.5 u.u) +- phi_k w 3 e.u
        const float2 x_even = fma2(mul(eu, A[c]), eu, B[c]);
        const float2 x_odd = mul(eu, Tc[c]);
        const float2 F = mul(en, Fw[c]);
        // minus the non-equilibrium, q_i - (phi_k - phi_ref) w_i - (velocity terms),
        // then q*_i = q_i + F_i - omega (minus the non-equilibrium)
        const float2 ma = sub(fma2(phin, -w, hv[i]), add(x_even, x_odd));
        const float2 mb = sub(fma2(phin, -w, hv[i + 1]), sub(x_even, x_odd));
        float2 a = fma2(ma, -om, add(hv[i], F));
        float2 b = fma2(mb, -om, sub(hv[i + 1], F));
        if constexpr (PMRT) {  // + w_i e_i . (3 (1 - omega_phi) J), odd in e
            float2 corr = bc(0.f);
            if (e.x) corr = acc_signed(corr, cJx, e.x);
            if (e.y) corr = acc_signed(corr, cJy, e.y);
            if (e.z) corr = acc_signed(corr, cJz, e.z);
            corr = mul(corr, w);
            a = add(a, corr);
            b = sub(b, corr);
        }
        const P qa = pack<T>(a), qb = pack<T>(b);
        store_pop<T, QP, H_SW, EDGE>(lh, n, i, qa);
        store_pop<T, QP, H_SW, EDGE>(lh, n, i + 1, qb);
        // the mass increments q*_i - q_i, exact in FP32 (differences of 16-bit values)
        if constexpr (!F32 && LBM_PAIR_MIXED) dsum = add(dsum, add(msub2<T>(qa, hv[i]), msub2<T>(qb, hv[i + 1])));
        else dsum = add(dsum, add(sub(unpack<T>(qa), hv[i]), sub(unpack<T>(qb), hv[i + 1])));
    }
    store_rest(lh.rest, n, sub(hv[0], dsum));
}

// One tile of 2 TXT x TYT x TZT cells (TXT x TYT x TZT threads).  The phi tile
// rows hold 2 TXT + 4 floats: columns 1 .. 2 TXT + 2 are x0 - 1 .. x0 + 2 TXT.
template <int TXT, int TYT, int TZT>
struct PairShape {
    static constexpr int PXT = 2 * TXT, ROWT = 2 * TXT + 4, NT = TXT * TYT * TZT;
};

template <typename T, int QG, int QP, bool G_SW, bool H_SW, int EDGE, int TXT, int TYT, int TZT, bool PMRT = false,
          bool W64 = false>
__device__ __forceinline__ void pair_cells(const Params &p, const Lat<T, W64> &lh, const Lat<T, W64> &lg, const Nb4 &n,
                                           bool active, const float *__restrict__ phi_in,
                                           float (*tile)[TYT + 2][2 * TXT + 4], float *__restrict__ phi_out,
                                           int *__restrict__ flag, int bx, int by, int bz, int tx, int ty, int tz) {
    using Sh = PairShape<TXT, TYT, TZT>;
    // the D2Q9 pair (nx x ny x 1 box): only the cells' own plane, kept as tile[1]
    constexpr bool PLANE = QP == 9;
    constexpr int HY = TYT + 2, HZ = TZT + 2, NROW = PLANE ? HY : HY * HZ;
    const bool wx = p.wall & 1, wy = p.wall & 2, wz = p.wall & 4;
    // phi^{k-1} rows of the tile with a one-cell halo (periodic wrap or wall
    // mirror per axis; coordinates past a ragged box end are clamped into the box,
    // those entries only feed inactive threads), loaded ahead of the populations
    constexpr int W = Sh::PXT + 2;  // x0 - 1 .. x0 + 2 TXT
    constexpr int NWARP = Sh::NT / 32;
    constexpr int EPT = TXT == 32 ? (NROW + NWARP - 1) / NWARP * 3 : (NROW * W + Sh::NT - 1) / Sh::NT;
    float tv[EPT];
    // row r of the tile: (kz, ky) = (r / HY, r % HY), or (1, r) in a plane
    auto row_kz = [&](int r) { return PLANE ? 1 : r / HY; };
    auto row_ky = [&](int r) { return PLANE ? r : r - (r / HY) * HY; };
    auto row_ptr = [&](int r) {
        const int kz = row_kz(r), ky = row_ky(r);
        const int gy = min(wrap_or_clamp(by * TYT - 1 + ky, p.ny, wy), p.ny - 1);
        const int gz = PLANE ? bz : min(wrap_or_clamp(bz * TZT - 1 + kz, p.nz, wz), p.nz - 1);
        return phi_in + (size_t)gy * p.nx + (size_t)gz * p.nx * p.ny;
    };
    auto gx = [&](int k) { return min(wrap_or_clamp(bx * Sh::PXT - 1 + k, p.nx, wx), p.nx - 1); };
    if constexpr (TXT == 32) {
        // warp w loads rows w, w + NWARP, ...; lane l the columns l, 32 + l and (l < 2) 64 + l
        const int lane = tx, warp = ty + TYT * tz;
        const int g0 = gx(lane), g1 = gx(32 + lane), g2 = gx(64 + lane);
#pragma unroll
        for (int j = 0; j < EPT / 3; ++j) {
            const int r = warp + j * NWARP;
            if (r < NROW) {
                const float *row = row_ptr(r);
                tv[3 * j] = __ldg(row + g0);
                tv[3 * j + 1] = __ldg(row + g1);
                if (lane < 2) tv[3 * j + 2] = __ldg(row + g2);
            }
        }
    } else {
        // element e = r W + k of the rows, consecutive threads on consecutive columns
        const int tid = tx + TXT * (ty + TYT * tz);
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            const int e = tid + j * Sh::NT;
            if (e < NROW * W) tv[j] = __ldg(row_ptr(e / W) + gx(e % W));
        }
    }
    using P = typename PairOf<T>::P;
    P gq[QG], hq[QP];
    float2 grest, hrest;
    if (active) {
        grest = load_rest(lg.rest, n);
#pragma unroll
        for (int i = 1; i < QG; ++i) gq[i] = load_pop<T, QG, G_SW, EDGE>(lg, n, i);
        hrest = load_rest(lh.rest, n);
#pragma unroll
        for (int i = 1; i < QP; ++i) hq[i] = load_pop<T, QP, H_SW, EDGE>(lh, n, i);
    }
    if constexpr (TXT == 32) {
        const int lane = tx, warp = ty + TYT * tz;
#pragma unroll
        for (int j = 0; j < EPT / 3; ++j) {
            const int r = warp + j * NWARP;
            if (r < NROW) {
                const int kz = row_kz(r), ky = row_ky(r);
                tile[kz][ky][1 + lane] = tv[3 * j];
                tile[kz][ky][33 + lane] = tv[3 * j + 1];
                if (lane < 2) tile[kz][ky][65 + lane] = tv[3 * j + 2];
            }
        }
    } else {
        const int tid = tx + TXT * (ty + TYT * tz);
#pragma unroll
        for (int j = 0; j < EPT; ++j) {
            const int e = tid + j * Sh::NT;
            if (e < NROW * W) {
                const int r = e / W, k = e - r * W;
                tile[row_kz(r)][row_ky(r)][1 + k] = tv[j];
            }
        }
    }
    __syncthreads();
    if (!active) return;
    float2 phic;
    const Stencil2 S = stencil_from_tile<PLANE>(
        [&](int dy, int dz) { return &tile[PLANE ? 1 : tz + 1 + dz][ty + 1 + dy][2 * tx]; }, phic);
    collide2<T, QG, QP, G_SW, H_SW, EDGE, PMRT, W64>(p, lh, lg, n, grest, gq, hrest, hq, S, phic, phi_out, flag);
}

// One tile (bx, by, bz) of 2 TXT x TYT x TZT cells of a box, one thread per pair
// of cells: per-thread offsets, then the bounce-back-checking path only if the
// tile touches a walled face (XONLY: a tile that touches only the x walls tests
// those alone, as the batch's walled boxes at most 64 cells wide mostly need).
// Every thread of the block must call this (it synchronises).
template <typename T, int QG, int QP, bool G_SW, bool H_SW, int TXT = TX, int TYT = TY, int TZT = TZ,
          bool XONLY = false, bool PMRT = false, bool W64 = false>
__device__ __forceinline__ void pair_tile(const Params &p, const Lat<T, W64> &lh, const Lat<T, W64> &lg,
                                          const float *__restrict__ phi_in, float *__restrict__ phi_out,
                                          int *__restrict__ flag, float (*tile)[TYT + 2][2 * TXT + 4], int bx,
                                          int by, int bz) {
    constexpr int PXT = 2 * TXT;
    const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
    const int x = bx * PXT + 2 * tx, y = by * TYT + ty, z = bz * TZT + tz;
    const bool active = x < p.nx && y < p.ny && z < p.nz;  // nx even: x + 1 < nx as well

    const bool wx = p.wall & 1, wy = p.wall & 2, wz = p.wall & 4;
    const int xc = min(x, p.nx - 2), yc = min(y, p.ny - 1), zc = min(z, p.nz - 1);
    const int nxy = p.nx * p.ny;
    const int c = xc + p.nx * yc + nxy * zc;
    Nb4 n;
    n.X[0] = c + wrap_or_clamp(xc - 1, p.nx, wx) - xc;
    n.X[1] = c;
    n.X[2] = c + 1;
    n.X[3] = c + wrap_or_clamp(xc + 2, p.nx, wx) - xc;
    n.Y[0] = (wrap_or_clamp(yc - 1, p.ny, wy) - yc) * p.nx;
    n.Y[1] = 0;
    n.Y[2] = (wrap_or_clamp(yc + 1, p.ny, wy) - yc) * p.nx;
    n.Z[0] = (wrap_or_clamp(zc - 1, p.nz, wz) - zc) * nxy;
    n.Z[1] = 0;
    n.Z[2] = (wrap_or_clamp(zc + 1, p.nz, wz) - zc) * nxy;
    const int lyz = (wy && yc == 0 ? 2 : 0) | (wz && zc == 0 ? 4 : 0);
    const int hyz = (wy && yc == p.ny - 1 ? 2 : 0) | (wz && zc == p.nz - 1 ? 4 : 0);
    n.lo[0] = lyz | (wx && xc == 0 ? 1 : 0);
    n.hi[0] = hyz;
    n.lo[1] = lyz;
    n.hi[1] = hyz | (wx && xc + 1 == p.nx - 1 ? 1 : 0);

    const bool ex = wx && (bx == 0 || (bx + 1) * PXT >= p.nx), ey = wy && (by == 0 || (by + 1) * TYT >= p.ny),
               ez = wz && (bz == 0 || (bz + 1) * TZT >= p.nz);
    if (!(ex || ey || ez))
        pair_cells<T, QG, QP, G_SW, H_SW, 0, TXT, TYT, TZT, PMRT, W64>(p, lh, lg, n, active, phi_in, tile, phi_out, flag, bx,
                                                            by, bz, tx, ty, tz);
    else if (XONLY && !(ey || ez))
        pair_cells<T, QG, QP, G_SW, H_SW, 1, TXT, TYT, TZT, PMRT, W64>(p, lh, lg, n, active, phi_in, tile, phi_out, flag, bx,
                                                            by, bz, tx, ty, tz);
    else
        pair_cells<T, QG, QP, G_SW, H_SW, 7, TXT, TYT, TZT, PMRT, W64>(p, lh, lg, n, active, phi_in, tile, phi_out, flag, bx,
                                                            by, bz, tx, ty, tz);
}

}  // namespace pairstep
}  // namespace lbm
