// lbm_device.cuh -- device building blocks of the coupled conservative
// Allen-Cahn LBM step (arXiv 2012.06144, Section 3) for sm_103a.
//
// Storage: one in-place copy per lattice, structure of arrays (plane i =
// direction i), streamed with the AA access pattern.  A lattice is either in
// natural layout (plane i at cell x holds f_i(x), pre-collision) or in swapped
// layout (plane opp(i) at x holds the post-collision f*_i(x) that still has to
// move to x + e_i).  A step on a natural lattice reads f_i(x) from (i, x) and
// writes f*_i(x) to (opp(i), x); a step on a swapped lattice reads f_i(x) from
// (opp(i), x - e_i) and writes f*_i(x) to (i, x + e_i).  Every thread reads and
// writes exactly the same locations, so the update is race-free in place.
// Walls use half-way bounce-back: a population whose source x - e_i (or
// destination x + e_i) lies beyond a walled face is read from (i, x) (written
// to (opp(i), x)) instead.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstddef>
#include <cstdint>
#include <type_traits>

namespace lbm {

struct V3 {
    int x, y, z;
};

// D3Q27 velocities in the documented numbering: rest, faces, edges, corners,
// each moving direction followed by its opposite.
__host__ __device__ constexpr V3 vel27(int i) {
    switch (i) {
        case 0: return {0, 0, 0};
        case 1: return {1, 0, 0};
        case 2: return {-1, 0, 0};
        case 3: return {0, 1, 0};
        case 4: return {0, -1, 0};
        case 5: return {0, 0, 1};
        case 6: return {0, 0, -1};
        case 7: return {1, 1, 0};
        case 8: return {-1, -1, 0};
        case 9: return {1, -1, 0};
        case 10: return {-1, 1, 0};
        case 11: return {1, 0, 1};
        case 12: return {-1, 0, -1};
        case 13: return {1, 0, -1};
        case 14: return {-1, 0, 1};
        case 15: return {0, 1, 1};
        case 16: return {0, -1, -1};
        case 17: return {0, 1, -1};
        case 18: return {0, -1, 1};
        case 19: return {1, 1, 1};
        case 20: return {-1, -1, -1};
        case 21: return {1, 1, -1};
        case 22: return {-1, -1, 1};
        case 23: return {1, -1, 1};
        case 24: return {-1, 1, -1};
        case 25: return {-1, 1, 1};
        default: return {1, -1, -1};
    }
}

// D3Q15 = rest, six faces, eight corners; D3Q19 = first 19 of D3Q27; D2Q9 = rest,
// the four x, y faces and the four xy edges (the two-dimensional pair).
template <int Q>
__host__ __device__ constexpr V3 vel(int i) {
    return (Q == 15 && i >= 7) ? vel27(i + 12) : (Q == 9 && i >= 5) ? vel27(i + 2) : vel27(i);
}

__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

// D3Q27 index of the direction (x, y, z) in {-1, 0, 1}^3
__host__ __device__ constexpr int idx27(int x, int y, int z) {
    for (int i = 0; i < 27; ++i) {
        const V3 e = vel27(i);
        if (e.x == x && e.y == y && e.z == z) return i;
    }
    return -1;
}

// Lattice weights selected by |e|^2.
template <int Q>
__host__ __device__ constexpr float wgt(int i) {
    const V3 e = vel<Q>(i);
    const int e2 = e.x * e.x + e.y * e.y + e.z * e.z;
    if (Q == 9) return e2 == 0 ? 4.0f / 9.0f : (e2 == 1 ? 1.0f / 9.0f : 1.0f / 36.0f);
    if (Q == 15) return e2 == 0 ? 2.0f / 9.0f : (e2 == 1 ? 1.0f / 9.0f : 1.0f / 72.0f);
    if (Q == 19) return e2 == 0 ? 1.0f / 3.0f : (e2 == 1 ? 1.0f / 18.0f : 1.0f / 36.0f);
    return e2 == 0 ? 8.0f / 27.0f : (e2 == 1 ? 2.0f / 27.0f : (e2 == 2 ? 1.0f / 54.0f : 1.0f / 216.0f));
}

// ---------------------------------------------------------------------------
// Population storage.  Every lattice is one rest plane in FP32 followed by q-1
// planes of its moving populations in a storage type T: float, __half or
// __nv_bfloat16.  A moving population f_i is kept as (f_i - w_i ref) * scale
// with a per-field shift ref and a power-of-two scale; the stored value decodes
// back exactly as w_i ref + q / scale.  With T = float, ref = 0 and scale = 1.
template <typename T>
__device__ __forceinline__ float to_f(T v) {
    if constexpr (std::is_same<T, __half>::value) return __half2float(v);
    else if constexpr (std::is_same<T, __nv_bfloat16>::value) return __bfloat162float(v);
    else return v;
}

template <typename T>
__device__ __forceinline__ T from_f(float v) {
    if constexpr (std::is_same<T, __half>::value) return __float2half_rn(v);
    else if constexpr (std::is_same<T, __nv_bfloat16>::value) return __float2bfloat16_rn(v);
    else return v;
}

// Kernel-side copy of the problem (derived in lbm_create).
struct Params {
    int nx, ny, nz;
    int wall;  // bit a set: axis a has walls on both faces
    long long N;
    float rho_L, drho;  // rho = rho_L + phi * (rho_H - rho_L)        (eq:density)
    float tau_L, dtau;  // tau = tau_L + phi * (tau_H - tau_L)
    float omega_phi;    // 1 / (tau_phi + 1/2), tau_phi = M / c_s^2
    float beta4;        // 4 beta, beta = 12 sigma / xi
    float kappa;        // 3 sigma xi / 2
    float inv_xi;
    float gx, gy, gz, rho_ref;
    float phi_lo, phi_hi;  // phi is clamped to [phi_lo, phi_hi] inside rho and tau
    // reduced-precision storage of the moving populations (ignored for FP32):
    // h_i stored as h_i - w_i h_ref, g_i stored as g_i * g_scale
    float h_ref, g_scale, g_inv_scale;
    int phase_mrt;  // 1: MRT phase collision (selects the kernel instance on the host)
    int step_form;  // fused step variant: 0 the library's choice, 2 one cell per thread, 3 two cells
};

// One lattice as seen by the auxiliary kernels: slot 0 (rest) in FP32, slot s >= 1
// at mov[(s - 1) N] in type T.
template <typename T>
struct LatView {
    float *rest;
    T *mov;
    long long N;
    float ref, scale, inv_scale;

    template <int Q>
    __device__ __forceinline__ float load(size_t slot, int dir, size_t idx) const {
        if (slot == 0) return rest[idx];
        const T q = mov[(slot - 1) * N + idx];
        if constexpr (std::is_same<T, float>::value) return q;
        else return fmaf(to_f(q), inv_scale, wgt<Q>(dir) * ref);
    }
    // stores v (already a value that encodes exactly, or any value for slot 0)
    template <int Q>
    __device__ __forceinline__ void store(size_t slot, int dir, size_t idx, float v) const {
        if (slot == 0) rest[idx] = v;
        else if constexpr (std::is_same<T, float>::value) mov[(slot - 1) * N + idx] = v;
        else mov[(slot - 1) * N + idx] = from_f<T>((v - wgt<Q>(dir) * ref) * scale);
    }
};

// Per-thread geometry: neighbour offsets along each axis (periodic wrap, or
// clamp at a walled face, which is the mirrored ghost value for phi) and the
// walled faces the cell touches.
struct Cell {
    int c;
    int xo[3], yo[3], zo[3];
    int lo, hi;  // bit a: cell on the low / high walled face of axis a
};

__device__ __forceinline__ int wrap_or_clamp(int v, int n, bool walled) {
    if (v < 0) return walled ? 0 : n - 1;
    if (v >= n) return walled ? n - 1 : 0;
    return v;
}

__device__ __forceinline__ Cell make_cell(const Params &p, int x, int y, int z) {
    Cell C;
    const bool wx = p.wall & 1, wy = p.wall & 2, wz = p.wall & 4;
    const int nxy = p.nx * p.ny;
    C.c = x + p.nx * (y + p.ny * z);
    C.xo[0] = wrap_or_clamp(x - 1, p.nx, wx);
    C.xo[1] = x;
    C.xo[2] = wrap_or_clamp(x + 1, p.nx, wx);
    C.yo[0] = wrap_or_clamp(y - 1, p.ny, wy) * p.nx;
    C.yo[1] = y * p.nx;
    C.yo[2] = wrap_or_clamp(y + 1, p.ny, wy) * p.nx;
    C.zo[0] = wrap_or_clamp(z - 1, p.nz, wz) * nxy;
    C.zo[1] = z * nxy;
    C.zo[2] = wrap_or_clamp(z + 1, p.nz, wz) * nxy;
    C.lo = (wx && x == 0 ? 1 : 0) | (wy && y == 0 ? 2 : 0) | (wz && z == 0 ? 4 : 0);
    C.hi = (wx && x == p.nx - 1 ? 1 : 0) | (wy && y == p.ny - 1 ? 2 : 0) | (wz && z == p.nz - 1 ? 4 : 0);
    return C;
}

__device__ __forceinline__ int nbr(const Cell &C, int dx, int dy, int dz) {
    return C.xo[dx + 1] + C.yo[dy + 1] + C.zo[dz + 1];
}

// True if x - e (sign = -1) or x + e (sign = +1) leaves the box through a wall.
__device__ __forceinline__ bool leaves(const Cell &C, V3 e, int sign) {
    const int ex = e.x * sign, ey = e.y * sign, ez = e.z * sign;
    return (ex > 0 && (C.hi & 1)) || (ex < 0 && (C.lo & 1)) || (ey > 0 && (C.hi & 2)) || (ey < 0 && (C.lo & 2)) ||
           (ez > 0 && (C.hi & 4)) || (ez < 0 && (C.lo & 4));
}

// Location (plane, cell) holding the pre-collision f_i(x) of a lattice.
template <int Q, bool SWAPPED>
__device__ __forceinline__ size_t pop_src(const Cell &C, long long N, int i) {
    if (!SWAPPED) return (size_t)i * N + C.c;
    const V3 e = vel<Q>(i);
    if (leaves(C, e, -1)) return (size_t)i * N + C.c;
    return (size_t)opp(i) * N + nbr(C, -e.x, -e.y, -e.z);
}

// The same location as (slot, element).
template <int Q, bool SWAPPED>
__device__ __forceinline__ void pop_src_loc(const Cell &C, int i, int &slot, int &idx) {
    if (!SWAPPED) {
        slot = i;
        idx = C.c;
        return;
    }
    const V3 e = vel<Q>(i);
    if (leaves(C, e, -1)) {
        slot = i;
        idx = C.c;
        return;
    }
    slot = opp(i);
    idx = nbr(C, -e.x, -e.y, -e.z);
}

// The 3x3x3 neighbourhood of phi, nb[(dz+1)*9 + (dy+1)*3 + (dx+1)].
__device__ __forceinline__ void gather_phi(const float *__restrict__ phi, const Cell &C, float nb[27]) {
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) nb[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)] = __ldg(phi + nbr(C, dx, dy, dz));
}

template <int Q>
__device__ __forceinline__ float nb_at(const float nb[27], int i) {
    const V3 e = vel<Q>(i);
    return nb[(e.z + 1) * 9 + (e.y + 1) * 3 + (e.x + 1)];
}

// Isotropic stencils eq:grad and eq:lap from the 3x3x3 neighbourhood.  The 26
// differences d(e) = phi(x + e) - phi(x) are formed once (exact in FP32 for
// neighbouring values) and grouped by opposite pairs and weight class (face,
// edge, corner), so that
//   grad phi = (1/c_s^2) sum_i w_i e_i phi(x + e_i) = 3 sum_class w_class D_class
//   lap  phi = (2/c_s^2) sum_i w_i d(e_i)           = 6 sum_class w_class L_class
// for D3Q15 (faces, corners), D3Q19 (faces, edges) and D3Q27 (all three) alike.
// A symmetric neighbourhood gives a gradient of exactly zero.
struct Stencil {
    float D1[3], D2[3], D3[3];  // sum over the class of e_a (phi(x + e) - phi(x - e)), one rep. per pair
    float L1, L2, L3;           // sum over the class of d(e) + d(-e)
};

// PLANE: the in-plane neighbours only (the D2Q9 pair on an nx x ny x 1 box).
template <bool PLANE = false>
__device__ __forceinline__ Stencil stencil_sums(const float nb[27]) {
    Stencil S;
#pragma unroll
    for (int a = 0; a < 3; ++a) S.D1[a] = S.D2[a] = S.D3[a] = 0.f;
    S.L1 = S.L2 = S.L3 = 0.f;
    const float c = nb[13];
#pragma unroll
    for (int i = 1; i < 27; i += 2) {  // i + 1 is the opposite of i
        const V3 e = vel27(i);
        if (PLANE && e.z != 0) continue;
        const float vp = nb_at<27>(nb, i), vm = nb_at<27>(nb, i + 1);
        const float D = vp - vm, L = (vp - c) + (vm - c);
        const int cls = e.x * e.x + e.y * e.y + e.z * e.z;
        float *Dc = cls == 1 ? S.D1 : (cls == 2 ? S.D2 : S.D3);
        if (e.x) Dc[0] += e.x > 0 ? D : -D;
        if (e.y) Dc[1] += e.y > 0 ? D : -D;
        if (e.z) Dc[2] += e.z > 0 ? D : -D;
        if (cls == 1) S.L1 += L;
        else if (cls == 2) S.L2 += L;
        else S.L3 += L;
    }
    return S;
}

// weight of a class (|e|^2 = 1, 2, 3) in lattice Q; 0 if the class is absent
template <int Q>
__host__ __device__ constexpr float wclass(int cls) {
    return Q == 9    ? (cls == 1 ? 1.0f / 9.0f : (cls == 2 ? 1.0f / 36.0f : 0.0f))
         : Q == 15 ? (cls == 1 ? 1.0f / 9.0f : (cls == 3 ? 1.0f / 72.0f : 0.0f))
         : Q == 19 ? (cls == 1 ? 1.0f / 18.0f : (cls == 2 ? 1.0f / 36.0f : 0.0f))
                   : (cls == 1 ? 2.0f / 27.0f : (cls == 2 ? 1.0f / 54.0f : 1.0f / 216.0f));
}

template <int Q>
__device__ __forceinline__ void stencil_grad(const Stencil &S, float &gx, float &gy, float &gz) {
    constexpr float w1 = 3.f * wclass<Q>(1), w2 = 3.f * wclass<Q>(2), w3 = 3.f * wclass<Q>(3);
    gx = w1 * S.D1[0] + (w2 != 0.f ? w2 * S.D2[0] : 0.f) + (w3 != 0.f ? w3 * S.D3[0] : 0.f);
    gy = w1 * S.D1[1] + (w2 != 0.f ? w2 * S.D2[1] : 0.f) + (w3 != 0.f ? w3 * S.D3[1] : 0.f);
    gz = w1 * S.D1[2] + (w2 != 0.f ? w2 * S.D2[2] : 0.f) + (w3 != 0.f ? w3 * S.D3[2] : 0.f);
}

template <int Q>
__device__ __forceinline__ float stencil_lap(const Stencil &S) {
    constexpr float w1 = 6.f * wclass<Q>(1), w2 = 6.f * wclass<Q>(2), w3 = 6.f * wclass<Q>(3);
    return w1 * S.L1 + (w2 != 0.f ? w2 * S.L2 : 0.f) + (w3 != 0.f ? w3 * S.L3 : 0.f);
}

// Macroscopic quantities and forces of the hydrodynamic step at one cell
// (Section 3.2).  Input: the pre-collision g_i(x) and the phi neighbourhood.
template <int QG>
struct Hydro {
    float pstar, ux, uy, uz;   // p* and u (eq:updateVelocityField)
    float Fx, Fy, Fz;          // total force (eq:forceHydro)
    float half_inv_rho;        // 1 / (2 rho)
    float s_nu;
    float a2xx, a2yy, a2zz, a2xy, a2xz, a2yz;  // Hermite second moments sum g (e e - c_s^2 I)
    float rho;
};

// SCALED: gv holds the populations multiplied by p.g_scale (a power of two, the
// 16-bit storage units); the moment sums are taken in those units and brought
// back with one multiplication each, which is exact.
// CASCADE (D3Q27): the moments by sums along x, then y, then z -- 66 additions
// instead of 111 over opposite pairs.  Same GPU, same process, 512^3: +2.7 % for
// the issue-bound FP16 step, but -5.3 % for FP32 and -1.0 % for BF16 (register
// allocation), so only the FP16 step takes it.
template <int QG, bool SCALED = false, bool CASCADE = false>
__device__ __forceinline__ void hydro_macro(const Params &p, const float gv[QG], float phi, const Stencil &S,
                                            Hydro<QG> &H) {
    // moments of g over opposite pairs: s = g_i + g_opp(i) carries the even
    // moments (p*, second moments), d = g_i - g_opp(i) the odd ones (j)
    float ps = gv[0], jx = 0.f, jy = 0.f, jz = 0.f, mxx = 0.f, myy = 0.f, mzz = 0.f, mxy = 0.f, mxz = 0.f,
          myz = 0.f;
    if constexpr (QG == 27 && CASCADE) {
        // D3Q27 spans {-1, 0, 1}^3: the moments up to second order by sums along x,
        // then y, then z
        float X0[3][3], X1[3][3], X2[3][3];  // per (z, y) line: sum, first and second moment in x
#pragma unroll
        for (int z = 0; z < 3; ++z)
#pragma unroll
            for (int y = 0; y < 3; ++y) {
                const float a = gv[idx27(-1, y - 1, z - 1)], b = gv[idx27(0, y - 1, z - 1)],
                            c = gv[idx27(1, y - 1, z - 1)];
                X2[z][y] = a + c;
                X0[z][y] = X2[z][y] + b;
                X1[z][y] = c - a;
            }
        float Y00[3], Y01[3], Y02[3], Y10[3], Y11[3], Y20[3];  // Yab: x-moment a, y-moment b, per z
#pragma unroll
        for (int z = 0; z < 3; ++z) {
            Y02[z] = X0[z][0] + X0[z][2];
            Y00[z] = Y02[z] + X0[z][1];
            Y01[z] = X0[z][2] - X0[z][0];
            Y10[z] = (X1[z][0] + X1[z][2]) + X1[z][1];
            Y11[z] = X1[z][2] - X1[z][0];
            Y20[z] = (X2[z][0] + X2[z][2]) + X2[z][1];
        }
        mzz = Y00[0] + Y00[2];
        ps = mzz + Y00[1];
        jz = Y00[2] - Y00[0];
        jy = (Y01[0] + Y01[2]) + Y01[1];
        myz = Y01[2] - Y01[0];
        myy = (Y02[0] + Y02[2]) + Y02[1];
        jx = (Y10[0] + Y10[2]) + Y10[1];
        mxz = Y10[2] - Y10[0];
        mxy = (Y11[0] + Y11[2]) + Y11[1];
        mxx = (Y20[0] + Y20[2]) + Y20[1];
    } else {
#pragma unroll
        for (int i = 1; i < QG; i += 2) {
            const V3 e = vel<QG>(i);
            const float s = gv[i] + gv[i + 1], d = gv[i] - gv[i + 1];
            ps += s;
            if (e.x) { jx += e.x > 0 ? d : -d; mxx += s; }
            if (e.y) { jy += e.y > 0 ? d : -d; myy += s; }
            if (e.z) { jz += e.z > 0 ? d : -d; mzz += s; }
            if (e.x && e.y) mxy += (e.x * e.y > 0) ? s : -s;
            if (e.x && e.z) mxz += (e.x * e.z > 0) ? s : -s;
            if (e.y && e.z) myz += (e.y * e.z > 0) ? s : -s;
        }
    }
    if constexpr (SCALED) {
        const float r = p.g_inv_scale;
        ps *= r;
        jx *= r;
        jy *= r;
        jz *= r;
        mxx *= r;
        myy *= r;
        mzz *= r;
        mxy *= r;
        mxz *= r;
        myz *= r;
    }
    float gpx, gpy, gpz;
    stencil_grad<QG>(S, gpx, gpy, gpz);
    const float lap = stencil_lap<QG>(S);

    const float phim = fminf(fmaxf(phi, p.phi_lo), p.phi_hi);
    const float rho = p.rho_L + phim * p.drho;  // eq:density
    const float hir = 0.5f * __frcp_rn(rho);
    const float tau = p.tau_L + phim * p.dtau;
    const float s_nu = __frcp_rn(tau + 0.5f);
    const float grx = p.drho * gpx, gry = p.drho * gpy, grz = p.drho * gpz;

    // eq:chemPot, eq:surfaceTension
    const float mu = p.beta4 * phi * (phi - 1.0f) * (phi - 0.5f) - p.kappa * lap;
    // eq:pressure_force, buoyancy
    const float cp = -ps * (1.0f / 3.0f);
    const float db = rho - p.rho_ref;
    const float f0x = mu * gpx + cp * grx + db * p.gx;
    const float f0y = mu * gpy + cp * gry + db * p.gy;
    const float f0z = mu * gpz + cp * grz + db * p.gz;

    // non-equilibrium second moments with u' (all forces but F_mu)
    const float upx = jx + f0x * hir, upy = jy + f0y * hir, upz = jz + f0z * hir;
    const float c3 = ps * (1.0f / 3.0f);
    // Hermite second moments over the lattice's own dimensions (no zz for D2Q9)
    const float a2xx = mxx - c3, a2yy = myy - c3, a2zz = QG == 9 ? 0.0f : mzz - c3;
    const float pxx = a2xx - upx * upx, pyy = a2yy - upy * upy, pzz = a2zz - upz * upz;
    const float pxy = mxy - upx * upy, pxz = mxz - upx * upz, pyz = myz - upy * upz;
    // eq:viscousForce: F_mu = -(nu / c_s^2) s_nu Pi_neq . grad rho = -tau s_nu Pi_neq . grad rho
    const float cm = -tau * s_nu;
    const float Fx = f0x + cm * (pxx * grx + pxy * gry + pxz * grz);
    const float Fy = f0y + cm * (pxy * grx + pyy * gry + pyz * grz);
    const float Fz = f0z + cm * (pxz * grx + pyz * gry + pzz * grz);

    H.pstar = ps;
    H.ux = jx + Fx * hir;
    H.uy = jy + Fy * hir;
    H.uz = jz + Fz * hir;
    H.Fx = Fx;
    H.Fy = Fy;
    H.Fz = Fz;
    H.half_inv_rho = hir;
    H.s_nu = s_nu;
    H.a2xx = a2xx;
    H.a2yy = a2yy;
    H.a2zz = a2zz;
    H.a2xy = mxy;
    H.a2xz = mxz;
    H.a2yz = myz;
    H.rho = rho;
}

// Post-collision population i of eq:improved_collision in Hermite form:
// zeroth moment p*, first moments u + F/(2 rho), second (Hermite) moments
// (1 - s_nu) a2 + s_nu u u, every higher moment 0.
template <int QG>
struct HydroPost {
    float m0, m1x, m1y, m1z, bxx, byy, bzz, bxy, bxz, byz, tr3;
};

template <int QG>
__device__ __forceinline__ HydroPost<QG> hydro_post(const Hydro<QG> &H) {
    HydroPost<QG> P;
    const float s = H.s_nu, r = 1.0f - s;
    P.m0 = H.pstar;
    P.m1x = 3.0f * (H.ux + H.Fx * H.half_inv_rho);
    P.m1y = 3.0f * (H.uy + H.Fy * H.half_inv_rho);
    P.m1z = 3.0f * (H.uz + H.Fz * H.half_inv_rho);
    const float bxx = r * H.a2xx + s * H.ux * H.ux;
    const float byy = r * H.a2yy + s * H.uy * H.uy;
    const float bzz = r * H.a2zz + s * H.uz * H.uz;
    P.bxx = 4.5f * bxx;
    P.byy = 4.5f * byy;
    P.bzz = 4.5f * bzz;
    P.bxy = 9.0f * (r * H.a2xy + s * H.ux * H.uy);
    P.bxz = 9.0f * (r * H.a2xz + s * H.ux * H.uz);
    P.byz = 9.0f * (r * H.a2yz + s * H.uy * H.uz);
    P.tr3 = 1.5f * (bxx + byy + bzz);  // 4.5 * trace / 3
    return P;
}

// The coefficients of hydro_post multiplied by s (a power of two: exact), so that
// hydro_gstar_pair returns s g*_i.
template <int QG>
__device__ __forceinline__ void scale_post(HydroPost<QG> &P, float s) {
    P.m0 *= s;
    P.m1x *= s;
    P.m1y *= s;
    P.m1z *= s;
    P.bxx *= s;
    P.byy *= s;
    P.bzz *= s;
    P.bxy *= s;
    P.bxz *= s;
    P.byz *= s;
    P.tr3 *= s;
}

// Even and odd parts of g*_i for a direction i of an opposite pair:
// g*_i = E + O, g*_opp(i) = E - O.
template <int QG>
__device__ __forceinline__ void hydro_gstar_pair(const HydroPost<QG> &P, int i, float &E, float &O) {
    const V3 e = vel<QG>(i);
    float ev = P.m0 - P.tr3, od = 0.f;
    if (e.x) { od += e.x > 0 ? P.m1x : -P.m1x; ev += P.bxx; }
    if (e.y) { od += e.y > 0 ? P.m1y : -P.m1y; ev += P.byy; }
    if (e.z) { od += e.z > 0 ? P.m1z : -P.m1z; ev += P.bzz; }
    if (e.x && e.y) ev += (e.x * e.y > 0) ? P.bxy : -P.bxy;
    if (e.x && e.z) ev += (e.x * e.z > 0) ? P.bxz : -P.bxz;
    if (e.y && e.z) ev += (e.y * e.z > 0) ? P.byz : -P.byz;
    E = wgt<QG>(i) * ev;
    O = wgt<QG>(i) * od;
}

}  // namespace lbm
