// lbm_step_impl.cuh -- device implementation of the fused coupled step, shared
// by the single-simulation kernel (lbm_step.cu) and the batched kernel
// (lbm_batch.cu).  See lbm_step.cu for the method and the layout of the work.
#pragma once

#include "lbm_internal.h"

namespace lbm {

#ifndef LBM_MIN_BLOCKS
#define LBM_MIN_BLOCKS 4  // resident blocks per SM the register budget is sized for
#endif

#ifndef LBM_TY
#define LBM_TY 2  // default tile: 32 x LBM_TY x LBM_TZ cells per block (32 x 2 x 4: fastest at 512^3)
#endif
#ifndef LBM_TZ
#define LBM_TZ 4
#endif
// Cache hints of the population loads and stores.  Loads: 0 plain, 1 evict-first
// (.cs), 2 read-only path (.nc: every location a thread reads is written only by
// the same thread, after the read, so no launch reads a value it wrote), 3 last
// use (.lu).  Stores: 0 plain (write-back), 1 evict-first (.cs).
#ifndef LBM_LOAD_HINT
#define LBM_LOAD_HINT 2  // 512^3, ms per step: .nc 7.52 (FP16 6.81), plain 7.52 (6.96), .cs 8.39
#endif
#ifndef LBM_STORE_HINT
#define LBM_STORE_HINT 0
#endif

constexpr int TX = 32;  // one warp = 32 consecutive x

// Plane pointers of both lattices: slot 0 (rest) is FP32, slots >= 1 hold the
// moving populations in the storage type of the launch.
struct Planes {
    void *h[27];
    void *g[27];
};

// Pairwise sum a[LO] + ... + a[LO + N - 1], halves first (a fixed association).
template <int LO, int N>
__device__ __forceinline__ float tree_sum(const float *a) {
    if constexpr (N == 1) return a[LO];
    else return tree_sum<LO, N / 2>(a) + tree_sum<LO + N / 2, N - N / 2>(a);
}

// Plane addresses of one lattice from a table of pointers (kernel parameters).
struct TableLat {
    void *const *t;
    template <typename U>
    __device__ __forceinline__ U *ptr(int s) const {
        return static_cast<U *>(t[s]);
    }
    template <typename U>
    __device__ __forceinline__ U *at(int s, int idx) const {
        return static_cast<U *>(t[s]) + idx;
    }
};

// Plane addresses of one lattice from its rest plane and first moving plane,
// with 32-bit element offsets (s - 1) N + idx into the moving planes (for boxes
// where 26 N < 2^32).
template <typename T>
struct BaseLat32 {
    float *rest;
    T *mov;
    unsigned N;
    template <typename U>
    __device__ __forceinline__ U *at(int s, int idx) const {
        if (s == 0) return reinterpret_cast<U *>(rest) + idx;
        return reinterpret_cast<U *>(mov) + ((unsigned)(s - 1) * N + (unsigned)idx);
    }
};

// Per-thread neighbour offsets: element index of (x+dx, y+dy, z+dz) is
// X[dx+1] + Y[dy+1] + Z[dz+1] (X includes the cell's own index).
struct Nb3 {
    int X[3], Y[3], Z[3];
    int lo, hi;  // walled faces touched by this cell (bit a: axis a)
};

__device__ __forceinline__ int nidx(const Nb3 &n, int dx, int dy, int dz) {
    return n.X[dx + 1] + n.Y[dy + 1] + n.Z[dz + 1];
}

// True if x + sign e leaves the box through a wall on one of the axes in AXES
// (bit a: axis a); the tile knows which walled faces it can touch.
template <int AXES>
__device__ __forceinline__ bool leaves3(const Nb3 &n, V3 e, int sign) {
    const int ex = e.x * sign, ey = e.y * sign, ez = e.z * sign;
    if constexpr (AXES == 1) return (ex > 0 && (n.hi & 1)) || (ex < 0 && (n.lo & 1));
    else
        return (ex > 0 && (n.hi & 1)) || (ex < 0 && (n.lo & 1)) || (ey > 0 && (n.hi & 2)) || (ey < 0 && (n.lo & 2)) ||
               (ez > 0 && (n.hi & 4)) || (ez < 0 && (n.lo & 4));
}

template <typename T>
__device__ __forceinline__ T ld_pop(const T *a) {
#if LBM_LOAD_HINT == 1
    return __ldcs(a);
#elif LBM_LOAD_HINT == 2
    return __ldg(a);
#elif LBM_LOAD_HINT == 3
    return __ldlu(a);
#else
    return *a;
#endif
}

template <typename T>
__device__ __forceinline__ void st_pop(T *a, T v) {
#if LBM_STORE_HINT == 1
    __stcs(a, v);
#else
    *a = v;
#endif
}

// Storage of the moving populations of one lattice in type T: the stored value q
// decodes as w_i ref + q inv_scale and encodes as (f - w_i ref) scale.
template <typename T>
struct Codec {
    float ref, scale, inv_scale;
    template <int Q>
    __device__ __forceinline__ float decode(T q, int i) const {
        if constexpr (std::is_same<T, float>::value) return q;
        else return fmaf(to_f(q), inv_scale, wgt<Q>(i) * ref);
    }
    template <int Q>
    __device__ __forceinline__ T encode(float f, int i) const {
        if constexpr (std::is_same<T, float>::value) return f;
        else return from_f<T>((f - wgt<Q>(i) * ref) * scale);
    }
};

// (slot, element) holding the pre-collision f_i(x) in the AA layout (see lbm_device.cuh)
template <int Q, bool SW, int EDGE>
__device__ __forceinline__ void src_loc(const Nb3 &n, int i, int &slot, int &idx) {
    if (!SW) {
        slot = i;
        idx = n.X[1];
        return;
    }
    const V3 e = vel<Q>(i);
    if (EDGE && leaves3<EDGE>(n, e, -1)) {
        slot = i;
        idx = n.X[1];
        return;
    }
    slot = opp(i);
    idx = nidx(n, -e.x, -e.y, -e.z);
}

// (slot, element) that receives the post-collision f*_i(x)
template <int Q, bool SW, int EDGE>
__device__ __forceinline__ void dst_loc(const Nb3 &n, int i, int &slot, int &idx) {
    if (!SW) {
        slot = opp(i);
        idx = n.X[1];
        return;
    }
    const V3 e = vel<Q>(i);
    if (EDGE && leaves3<EDGE>(n, e, +1)) {
        slot = opp(i);
        idx = n.X[1];
        return;
    }
    slot = i;
    idx = nidx(n, e.x, e.y, e.z);
}

template <typename T, int Q, bool SW, int EDGE, typename L>
__device__ __forceinline__ float pop_load(const L &lat, const Nb3 &n, int i, const Codec<T> &cd) {
    int slot, idx;
    src_loc<Q, SW, EDGE>(n, i, slot, idx);
    if (slot == 0) return ld_pop(lat.template at<float>(0, idx));
    return cd.template decode<Q>(ld_pop(lat.template at<T>(slot, idx)), i);
}

// FP16 storage: both lattices stay in their storage units through the step
// (g times g_scale, h_i minus w_i phi_ref), which removes a decode and an encode
// per population: +5.0 % at 512^3 in a same-GPU comparison.  BF16 keeps the
// decode-compute-encode form, which measured 9 % faster for it there.  The FP16
// step also takes the D3Q27 moments by the x-y-z cascade of hydro_macro.
template <typename T>
constexpr bool in_units() {
    return std::is_same<T, __half>::value;
}

// g_i in 16-bit storage units: the stored moving value as is, the FP32 rest
// population times the storage scale
template <typename T, int Q, bool SW, int EDGE, typename L>
__device__ __forceinline__ float pop_load_units(const L &lat, const Nb3 &n, int i, float scale) {
    int slot, idx;
    src_loc<Q, SW, EDGE>(n, i, slot, idx);
    if (slot == 0) return ld_pop(lat.template at<float>(0, idx)) * scale;
    return to_f(ld_pop(lat.template at<T>(slot, idx)));
}

// stores the rest population (i = 0, FP32) or an encoded moving population
template <typename T, int Q, bool SW, int EDGE, typename L>
__device__ __forceinline__ void pop_store_rest(const L &lat, const Nb3 &n, float v) {
    int slot, idx;
    dst_loc<Q, SW, EDGE>(n, 0, slot, idx);
    st_pop(lat.template at<float>(0, idx), v);
}

template <typename T, int Q, bool SW, int EDGE, typename L>
__device__ __forceinline__ void pop_store_enc(const L &lat, const Nb3 &n, int i, T q) {
    int slot, idx;
    dst_loc<Q, SW, EDGE>(n, i, slot, idx);
    st_pop(lat.template at<T>(slot, idx), q);
}

// Collision of both lattices at one cell and the streaming stores, from the
// pre-collision populations gv (g^{k-1}), hv (h^k) and the 3x3x3 neighbourhood nb
// of phi^{k-1}.
template <typename T, int QG, int QP, bool G_SW, bool H_SW, bool HYDRO, bool PMRT, int EDGE, typename LH,
          typename LG>
__device__ __forceinline__ void collide_and_store(const Params &p, const LH &lh, const LG &lg, const Nb3 &n, const float *gv,
                                                  const float *hv, const float *nb, float *__restrict__ phi_out,
                                                  int *__restrict__ flag) {
    const Codec<T> ch{p.h_ref, 1.0f, 1.0f}, cg{0.0f, p.g_scale, p.g_inv_scale};
    const float phic = nb[13];
    const Stencil S = stencil_sums<QP == 9>(nb);
    float ux = 0.f, uy = 0.f, uz = 0.f;

    // ---- hydrodynamic step k-1 (Section 3.2)
    if (HYDRO) {
        // FP16 storage: g arrives in storage units (g_scale, a power of two) and
        // the moments are brought back once; the post-collision coefficients are
        // scaled once, so E +- O below is already the value to store.
        constexpr bool UNITS = in_units<T>();
        Hydro<QG> Hd;
        hydro_macro<QG, UNITS, UNITS>(p, gv, phic, S, Hd);
        HydroPost<QG> P = hydro_post<QG>(Hd);
        if constexpr (UNITS) scale_post<QG>(P, p.g_scale);
        // The rest population takes p* - sum_{i>0} g*_i, with each g*_i as the next
        // reader will decode it, so the stored populations keep the zeroth moment
        // p* of eq:improved_collision to rounding (the FP32 weights do not sum to 1).
        float gsum = 0.f;
#pragma unroll
        for (int i = 1; i < QG; i += 2) {
            float E, O;
            hydro_gstar_pair<QG>(P, i, E, O);
            if constexpr (UNITS) {
                const T qa = from_f<T>(E + O), qb = from_f<T>(E - O);
                pop_store_enc<T, QG, G_SW, EDGE>(lg, n, i, qa);
                pop_store_enc<T, QG, G_SW, EDGE>(lg, n, i + 1, qb);
                gsum += to_f(qa) + to_f(qb);
            } else {
                const T qa = cg.template encode<QG>(E + O, i), qb = cg.template encode<QG>(E - O, i + 1);
                pop_store_enc<T, QG, G_SW, EDGE>(lg, n, i, qa);
                pop_store_enc<T, QG, G_SW, EDGE>(lg, n, i + 1, qb);
                gsum += cg.template decode<QG>(qa, i) + cg.template decode<QG>(qb, i + 1);
            }
        }
        if constexpr (UNITS) gsum *= p.g_inv_scale;
        pop_store_rest<T, QG, G_SW, EDGE>(lg, n, Hd.pstar - gsum);
        ux = Hd.ux;
        uy = Hd.uy;
        uz = Hd.uz;
        if (!(fabsf(Hd.pstar) < 1e30f)) *flag = 1;
    }

    // ---- phase-field step k (Section 3.1)
    // phi_k = sum_i h_i (eq:updatePhaseField), summed as a tree over opposite pairs
    // FP16 storage: the moving h_i arrive as q_i = h_i - w_i phi_ref and stay in
    // those units; sum_{i>0} w_i phi_ref enters phi_k once
    constexpr bool HU = in_units<T>();
    constexpr int NPR = (QP + 1) / 2;
    float pr[NPR];
    pr[0] = HU ? hv[0] + p.h_ref * (1.0f - wgt<QP>(0)) : hv[0];
#pragma unroll
    for (int j = 0; j < NPR - 1; ++j) pr[j + 1] = hv[2 * j + 1] + hv[2 * j + 2];
    const float phik = tree_sum<0, NPR>(pr);
    phi_out[n.X[1]] = phik;
    if (!(fabsf(phik) < 1e30f)) *flag = 1;

    // interface normal from eq:grad with the phase lattice's weights (the class
    // sums of the same neighbourhood)
    float Gx, Gy, Gz;
    stencil_grad<QP>(S, Gx, Gy, Gz);
    const float G2 = Gx * Gx + Gy * Gy + Gz * Gz;
    float nx = 0.f, ny = 0.f, nz = 0.f;
    if (G2 > 1e-24f) {
        float inv = rsqrtf(G2);
        inv = inv * (1.5f - 0.5f * G2 * inv * inv);  // one Newton step: no systematic bias in |n|
        nx = Gx * inv;
        ny = Gy * inv;
        nz = Gz * inv;
    }
    const float pc = phic - 0.5f;
    const float theta = (1.0f - 4.0f * pc * pc) * p.inv_xi;
    const float uu = 1.5f * (ux * ux + uy * uy + uz * uz);
    float om = p.omega_phi, fc = 1.0f - 0.5f * om;
    // MRT (Section 3.1, first-order moments relaxed with omega_phi, the rest with
    // 1, weighted-orthogonal basis): the SRT update with rate 1 plus
    // (1 - omega_phi) w_i e_i . J / c_s^2, J = sum_j e_j (h_j - h^eq_j + F_j / 2)
    //   = sum_j e_j h_j - phi_k u + theta c_s^2 n / 2.
    float cJx = 0.f, cJy = 0.f, cJz = 0.f;
    if constexpr (PMRT) {
        float jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
        for (int i = 1; i < QP; i += 2) {
            const V3 e = vel<QP>(i);
            const float dh = hv[i] - hv[i + 1];
            jx += e.x * dh;
            jy += e.y * dh;
            jz += e.z * dh;
        }
        const float c = 3.0f * (1.0f - om), th = theta * (0.5f / 3.0f);
        cJx = c * (fmaf(th, nx, jx) - phik * ux);
        cJy = c * (fmaf(th, ny, jy) - phik * uy);
        cJz = c * (fmaf(th, nz, jz) - phik * uz);
        om = 1.0f;
        fc = 0.5f;
    }
    // h*_i = h_i + omega (h^eq_i - h_i - F_i/2) + F_i over opposite pairs, with
    // h^eq = phi_k w (1 + 3 e.u + 4.5 (e.u)^2 - 1.5 u.u) and F_i = theta w e.n.
    // The non-equilibrium h^eq_i - h_i is formed as fma(phi_k, w, -h_i) + phi_k w
    // (velocity terms), so it carries no rounding of the large product phi w.
    // The rest population takes h_0 - sum_{i>0} (h*_i - h_i), with each h*_i as
    // the next reader will decode it: each increment is exact in FP32 (h*_i and
    // h_i are close), so the stored populations sum to the incoming sum_i h_i up
    // to the rounding of small increments, i.e. the cell's phase mass is kept.
    // in storage units h^eq_i - h_i = (phi_k - phi_ref) w_i - q_i + (velocity terms)
    const float phin = HU ? phik - p.h_ref : phik;
    float dsum = 0.f;
#pragma unroll
    for (int i = 1; i < QP; i += 2) {
        const V3 e = vel<QP>(i);
        const float w = wgt<QP>(i);
        const float eu = e.x * ux + e.y * uy + e.z * uz;
        const float en = e.x * nx + e.y * ny + e.z * nz;
        const float pw = phik * w;
        const float x_even = pw * (4.5f * eu * eu - uu);
        const float x_odd = pw * 3.0f * eu;
        const float F = fc * (theta * w * en);
        const float neq_a = fmaf(phin, w, -hv[i]) + (x_even + x_odd);
        const float neq_b = fmaf(phin, w, -hv[i + 1]) + (x_even - x_odd);
        float a = hv[i] + fmaf(om, neq_a, F);
        float b = hv[i + 1] + fmaf(om, neq_b, -F);
        if constexpr (PMRT) {
            const float corr = w * (e.x * cJx + e.y * cJy + e.z * cJz);
            a += corr;
            b -= corr;
        }
        if constexpr (HU) {
            const T qa = from_f<T>(a), qb = from_f<T>(b);
            pop_store_enc<T, QP, H_SW, EDGE>(lh, n, i, qa);
            pop_store_enc<T, QP, H_SW, EDGE>(lh, n, i + 1, qb);
            dsum += (to_f(qa) - hv[i]) + (to_f(qb) - hv[i + 1]);
        } else {
            const T qa = ch.template encode<QP>(a, i), qb = ch.template encode<QP>(b, i + 1);
            pop_store_enc<T, QP, H_SW, EDGE>(lh, n, i, qa);
            pop_store_enc<T, QP, H_SW, EDGE>(lh, n, i + 1, qb);
            dsum += (ch.template decode<QP>(qa, i) - hv[i]) + (ch.template decode<QP>(qb, i + 1) - hv[i + 1]);
        }
    }
    pop_store_rest<T, QP, H_SW, EDGE>(lh, n, hv[0] - dsum);
}

// ---------------------------------------------------------------------------
// The phi halo tile staged by the tensor-memory accelerator: one
// cp.async.bulk.tensor load of a (TX + 8) x (TY + 2) x (TZ + 2) box starting at
// (x0 - 4, y0 - 1, z0 - 1) (x0 - 4 keeps the copy on a 16-byte boundary; the
// tile row is 40 floats with cell x0 at offset 4), completed on an mbarrier.
// Coordinates outside the box read as 0: entries beyond a walled face are then
// mirrored in shared memory (phi(-1) = phi(0), the neutral wetting of the
// oracle), and tiles on a periodic face of the box are filled by per-thread
// loads instead (their halo wraps around).
constexpr int kTmaRow = TX + 8;
constexpr int kTmaWaitLimit = 1 << 20;  // try_wait polls before the copy counts as lost

struct HaloTma {
    uint64_t *bar;  // the block's mbarrier (phase 0 completes when the tile has landed)
    int *err;       // set to 1 if the copy did not complete within kTmaWaitLimit polls
};

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void tma_bar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// the arrival of the issuing thread with the byte count of the copy, then the copy
__device__ __forceinline__ void tma_load_tile(float *dst, const void *tensor_map, int x, int y, int z, uint64_t *bar,
                                              unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_addr(dst)),
        "l"(tensor_map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// bounded wait for phase 0 of the block's mbarrier
__device__ __forceinline__ bool tma_bar_wait(uint64_t *bar) {
    for (int k = 0; k < kTmaWaitLimit; ++k) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(smem_addr(bar))
            : "memory");
        if (done) return true;
    }
    return false;
}

// True if the tile's one-cell halo stays inside the box on every periodic axis
// (the copy cannot wrap); walled axes are mirrored after the copy.
template <int TY, int TZ>
__device__ __forceinline__ bool tma_halo_fits(const Params &p, int bx, int by, int bz) {
    const bool wx = p.wall & 1, wy = p.wall & 2, wz = p.wall & 4;
    const bool ix = bx > 0 && (bx + 1) * TX < p.nx, iy = by > 0 && (by + 1) * TY < p.ny,
               iz = bz > 0 && (bz + 1) * TZ < p.nz;
    return (wx || ix) && (wy || iy) && (wz || iz);
}

// Mirror of the halo entries beyond the walled faces the tile touches: each takes
// the value at its coordinates clamped into the box, an interior entry that the
// copy delivered and that no thread writes here.
template <int TY, int TZ, int HW>
__device__ __forceinline__ void mirror_walls(const Params &p, float (*tile)[TY + 2][HW], int bx, int by, int bz,
                                             int tid) {
    constexpr int OX = HW == TX + 2 ? 1 : 4, NT = TX * TY * TZ, WX = TX + 2;
    const bool wx = p.wall & 1, wy = p.wall & 2, wz = p.wall & 4;
    const int gx0 = bx * TX - OX, gy0 = by * TY - 1, gz0 = bz * TZ - 1;
    auto fix = [&](int kx, int ky, int kz) {
        const int gx = gx0 + kx, gy = gy0 + ky, gz = gz0 + kz;
        const int cx = wx ? min(max(gx, 0), p.nx - 1) : gx, cy = wy ? min(max(gy, 0), p.ny - 1) : gy,
                  cz = wz ? min(max(gz, 0), p.nz - 1) : gz;
        if (cx != gx || cy != gy || cz != gz) tile[kz][ky][kx] = tile[cz - gz0][cy - gy0][cx - gx0];
    };
    // x faces: the columns just outside the tile, every (y, z) row of the halo
    if (wx && (bx == 0 || (bx + 1) * TX >= p.nx))
        for (int e = tid; e < 2 * (TY + 2) * (TZ + 2); e += NT) {
            const int r = e >> 1, ky = r % (TY + 2), kz = r / (TY + 2);
            fix((e & 1) ? OX + min(TX, p.nx - bx * TX) : OX - 1, ky, kz);
        }
    // y faces and z faces: the rows / planes just outside, over the 34 needed columns
    if (wy && (by == 0 || (by + 1) * TY >= p.ny))
        for (int e = tid; e < 2 * WX * (TZ + 2); e += NT) {
            const int r = e / WX, kx = OX - 1 + (e - r * WX), kz = r >> 1;
            fix(kx, (r & 1) ? 1 + min(TY, p.ny - by * TY) : 0, kz);
        }
    if (wz && (bz == 0 || (bz + 1) * TZ >= p.nz))
        for (int e = tid; e < 2 * WX * (TY + 2); e += NT) {
            const int r = e / WX, kx = OX - 1 + (e - r * WX), ky = r >> 1;
            fix(kx, ky, (r & 1) ? 1 + min(TZ, p.nz - bz * TZ) : 0);
        }
}

template <typename T, int QG, int QP, bool G_SW, bool H_SW, bool HYDRO, bool PMRT, int EDGE, int TY, int TZ,
          int HW, typename LH, typename LG>
__device__ __forceinline__ void cell_update(const Params &p, const LH &lh, const LG &lg, const Nb3 &n, bool active,
                                            const float *__restrict__ phi_in, float (*tile)[TY + 2][HW],
                                            float *__restrict__ phi_out, int *__restrict__ flag, int bx, int by,
                                            int bz, int tx, int ty, int tz, const HaloTma *tma) {
    constexpr int HX = TX + 2, HY = TY + 2, HZ = TZ + 2;
    constexpr int OX = HW == TX + 2 ? 1 : 4;  // tile column of cell x0: 1 (34-float rows) or 4 (TMA rows)
    static_assert(HW == TX + 2 || HW == kTmaRow, "tile row width");
    // the D2Q9 pair (nx x ny x 1 box): only the cell's own plane, kept as tile[1]
    constexpr bool PLANE = QP == 9;

    // ---- phi^{k-1} tile with a one-cell halo (wrap on periodic axes, mirror at
    // walls), filled row by row: warp w loads rows w, w + 8, ... of the HZ x HY
    // rows, lane l the x-offsets l and (lanes 0, 1) 32 + l.  The loads are issued
    // before the population loads so that their latency overlaps.
    constexpr int NROW = PLANE ? HY : HY * HZ, NWARP = TX * TY * TZ / 32, RPW = (NROW + NWARP - 1) / NWARP;
    const int lane = tx, warp = ty + TY * tz;
    const bool wx = p.wall & 1, wy = p.wall & 2, wz = p.wall & 4;
    const int gx0 = min(wrap_or_clamp(bx * TX - 1 + lane, p.nx, wx), p.nx - 1);
    const int gx1 = min(wrap_or_clamp(bx * TX + 31 + lane, p.nx, wx), p.nx - 1);
    float tv0[RPW], tv1[RPW];
#pragma unroll
    for (int k = 0; k < RPW; ++k) {
        const int r = warp + k * NWARP;
        if (!tma && r < NROW) {
            const int kz = PLANE ? 1 : r / HY, ky = PLANE ? r : r - kz * HY;
            // coordinates beyond a ragged box end are clamped into the box; those
            // halo entries only feed threads that are inactive
            const int gy = min(wrap_or_clamp(by * TY - 1 + ky, p.ny, wy), p.ny - 1);
            const int gz = PLANE ? bz : min(wrap_or_clamp(bz * TZ - 1 + kz, p.nz, wz), p.nz - 1);
            const float *row = phi_in + (size_t)gy * p.nx + (size_t)gz * p.nx * p.ny;
            tv0[k] = __ldg(row + gx0);
            if (lane < HX - 32) tv1[k] = __ldg(row + gx1);
        }
    }

    // ---- the population loads
    const Codec<T> ch{p.h_ref, 1.0f, 1.0f}, cg{0.0f, p.g_scale, p.g_inv_scale};
    float gv[QG], hv[QP];
    if (active) {
        if (HYDRO) {
#pragma unroll
            for (int i = 0; i < QG; ++i)
                gv[i] = in_units<T>() ? pop_load_units<T, QG, G_SW, EDGE>(lg, n, i, p.g_scale)
                                      : pop_load<T, QG, G_SW, EDGE>(lg, n, i, cg);
        }
#pragma unroll
        for (int i = 0; i < QP; ++i)
            hv[i] = in_units<T>() ? pop_load_units<T, QP, H_SW, EDGE>(lh, n, i, 1.0f)
                                  : pop_load<T, QP, H_SW, EDGE>(lh, n, i, ch);
    }

    if (!tma) {
#pragma unroll
        for (int k = 0; k < RPW; ++k) {
            const int r = warp + k * NWARP;
            if (r < NROW) {
                const int kz = PLANE ? 1 : r / HY, ky = PLANE ? r : r - kz * HY;
                tile[kz][ky][OX - 1 + lane] = tv0[k];
                if (lane < HX - 32) tile[kz][ky][OX + 31 + lane] = tv1[k];
            }
        }
        __syncthreads();
    } else {
        // the copy issued at block start; then the mirror of walled faces, if any
        const bool landed = tma_bar_wait(tma->bar);
        const bool walls = (wx && (bx == 0 || (bx + 1) * TX >= p.nx)) || (wy && (by == 0 || (by + 1) * TY >= p.ny)) ||
                           (wz && (bz == 0 || (bz + 1) * TZ >= p.nz));
        if (walls) {
            if (__syncthreads_or(!landed)) {
                if (tx == 0 && ty == 0 && tz == 0) *tma->err = 1;
                return;
            }
            mirror_walls<TY, TZ, HW>(p, tile, bx, by, bz, tx + TX * (ty + TY * tz));
            __syncthreads();
        } else if (!landed) {
            *tma->err = 1;
            return;
        }
    }
    if (!active) return;
    float nb[27];
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx)
                nb[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)] = tile[PLANE ? 1 : tz + 1 + dz][ty + 1 + dy][tx + OX + dx];
    collide_and_store<T, QG, QP, G_SW, H_SW, HYDRO, PMRT, EDGE>(p, lh, lg, n, gv, hv, nb, phi_out, flag);
}

// One tile (bx, by, bz) of 32 x TY x TZ cells, one thread per cell: per-thread
// neighbour offsets, then the bounce-back-checking path only if the tile touches
// a walled face.  Every thread of the block must call this (it synchronises).
// XONLY: a tile that touches only the x walls takes a path that tests the x walls
// alone (the batched walled boxes, at most 64 cells wide, are mostly such tiles;
// for the single-simulation kernel the extra path cost more than it saved).
// HW / tma: the phi tile's row width (TX + 2, filled by per-thread loads; or
// kTmaRow, with tma given when the block has issued the tile's TMA copy).
template <typename T, int QG, int QP, bool G_SW, bool H_SW, bool HYDRO, bool PMRT, int TY, int TZ, bool XONLY = false,
          int HW = TX + 2, typename LH, typename LG>
__device__ __forceinline__ void tile_update(const Params &p, const LH &lh, const LG &lg,
                                            const float *__restrict__ phi_in, float *__restrict__ phi_out,
                                            int *__restrict__ flag, float (*tile)[TY + 2][HW], int bx, int by,
                                            int bz, int tx, int ty, int tz, const HaloTma *tma = nullptr) {
    const int x = bx * TX + tx;
    const int y = by * TY + ty;
    const int z = bz * TZ + tz;
    const bool active = x < p.nx && y < p.ny && z < p.nz;

    const bool wx = p.wall & 1, wy = p.wall & 2, wz = p.wall & 4;
    const int xc = min(x, p.nx - 1), yc = min(y, p.ny - 1), zc = min(z, p.nz - 1);
    const int nxy = p.nx * p.ny;
    Nb3 n;
    const int c = xc + p.nx * yc + nxy * zc;
    n.X[0] = c + wrap_or_clamp(xc - 1, p.nx, wx) - xc;
    n.X[1] = c;
    n.X[2] = c + wrap_or_clamp(xc + 1, p.nx, wx) - xc;
    n.Y[0] = (wrap_or_clamp(yc - 1, p.ny, wy) - yc) * p.nx;
    n.Y[1] = 0;
    n.Y[2] = (wrap_or_clamp(yc + 1, p.ny, wy) - yc) * p.nx;
    n.Z[0] = (wrap_or_clamp(zc - 1, p.nz, wz) - zc) * nxy;
    n.Z[1] = 0;
    n.Z[2] = (wrap_or_clamp(zc + 1, p.nz, wz) - zc) * nxy;
    n.lo = (wx && xc == 0 ? 1 : 0) | (wy && yc == 0 ? 2 : 0) | (wz && zc == 0 ? 4 : 0);
    n.hi = (wx && xc == p.nx - 1 ? 1 : 0) | (wy && yc == p.ny - 1 ? 2 : 0) | (wz && zc == p.nz - 1 ? 4 : 0);

    // the walled faces this tile touches, by axis: none (the plain path), the x walls
    // only (every tile of a walled box at most 64 cells wide), or any
    const bool ex = wx && (bx == 0 || (bx + 1) * TX >= p.nx), ey = wy && (by == 0 || (by + 1) * TY >= p.ny),
               ez = wz && (bz == 0 || (bz + 1) * TZ >= p.nz);
    if (!(ex || ey || ez))
        cell_update<T, QG, QP, G_SW, H_SW, HYDRO, PMRT, 0, TY, TZ, HW>(p, lh, lg, n, active, phi_in, tile, phi_out,
                                                                       flag, bx, by, bz, tx, ty, tz, tma);
    else if (XONLY && !(ey || ez))
        cell_update<T, QG, QP, G_SW, H_SW, HYDRO, PMRT, 1, TY, TZ, HW>(p, lh, lg, n, active, phi_in, tile, phi_out,
                                                                       flag, bx, by, bz, tx, ty, tz, tma);
    else
        cell_update<T, QG, QP, G_SW, H_SW, HYDRO, PMRT, 7, TY, TZ, HW>(p, lh, lg, n, active, phi_in, tile, phi_out,
                                                                       flag, bx, by, bz, tx, ty, tz, tma);
}

}  // namespace lbm
