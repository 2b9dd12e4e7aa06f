// lbm_batch.cu -- many independent simulations advanced together.
//
// A batch owns ordinary simulation handles (its members), which keep their own
// parameters, workspaces and time levels; initialisation, fields, reductions and
// state transfer go through the single-simulation entry points on a member.
// Stepping is shared: the members' tiles of 32 x TY x TZ cells are packed into
// one table and one launch per time step (per group of up to kGroup members)
// runs one block per table entry.  The per-tile work is exactly the
// single-simulation step (Algorithm 2, coupled phase-field and hydrodynamic
// update), so members evolve as they would alone.
//
// The members' descriptors (Section 3 parameters, lattice pointers, phi buffers)
// travel in the launch's own parameter block (__grid_constant__), so a block
// reads its member's values through the constant cache as the single-simulation
// kernel does; loading them into registers or from shared memory costs the
// register-bound step many spilled bytes.  A persistent form (each block looping
// over a chunk of the table) was tried and dropped: the loop around the step
// body makes ptxas spill 280-400 bytes per thread at 64-128 registers, against
// 24 bytes for one tile per block.
//
// Steps are replayed from CUDA graphs of kGraphSteps launches.  The autotuner
// times every tile shape and table order on the batch itself and keeps the
// fastest.
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "lbm_handle.h"
#include "lbm_pair_impl.cuh"

namespace lbm {

constexpr int kGroup = 64;  // members per launch: 64 descriptors and tensor-map pairs fit the 32 KB parameter block
constexpr int kGraphSteps = 16;

// A member's lattices are addressed as the single-simulation kernel addresses
// walled boxes: base pointers plus 32-bit plane offsets (every member passes
// offsets32), which measured 2.2% faster on the batched workload than a table
// of 42 plane pointers per member and keeps the descriptor small.
//
//
// The phi halo tile is staged either by per-thread loads or by one TMA copy per
// block (tensor maps of each member's two phi buffers for the current tile shape,
// also in the parameter block); the autotuner times both.
struct MemberDesc {
    Params p;
    float *h_rest, *h_mov, *g_rest, *g_mov;  // rest and first moving plane of each lattice
    float *phi[2];
    int *flag;  // [0] divergence, [1] a TMA halo copy that did not complete
};

struct GroupArgs {
    CUtensorMap phi_map[kGroup][2];  // phi[0], phi[1] as 3-D FP32 tensors, box kTmaRow x (TY + 2) x (TZ + 2)
    MemberDesc m[kGroup];
};
static_assert(sizeof(GroupArgs) + 32 <= 32764, "kernel parameter block limit");

// Tile shapes of the table: tx x ty x tz cells.  The first three run the one-cell
// step (a thread per cell); the last the two-cell step of lbm_pair_impl.cuh (a
// thread per pair of cells: 16 x 4 x 2 threads), for batches whose members all
// have nx even, with per-thread halo loads.  All are 32 cells wide, the width
// that keeps the tiles of the small walled boxes full.
struct TileShape {
    int ty, tz, tx;
};
constexpr int kPairTX = 16, kPairTY = 4, kPairTZ = 2;  // threads of the two-cell tile
constexpr TileShape kShapes[] = {{4, 2, TX}, {8, 1, TX}, {2, 4, TX}, {kPairTY, kPairTZ, 2 * kPairTX}};
constexpr int kNumShapes = 4;
constexpr int kPairShape = 3;
constexpr int kNumOrders = 2;  // 0: member after member, 1: members interleaved tile by tile
constexpr int kNumHalos = 2;   // 0: per-thread loads, 1: TMA copy (per-thread loads on periodic faces)

// One tile (member within the group, bx, by, bz) = e of the table.
template <int QG, bool G_SW, bool H_SW, int TY, int TZ, int HALO>
__device__ __forceinline__ void batch_tile(const GroupArgs &a, const int4 e, int cur,
                                           float (*tile)[TY + 2][HALO ? kTmaRow : TX + 2], uint64_t *bar) {
    constexpr int HW = HALO ? kTmaRow : TX + 2;
    const MemberDesc &d = a.m[e.x];
    const BaseLat32<float> lh{d.h_rest, d.h_mov, (unsigned)d.p.N}, lg{d.g_rest, d.g_mov, (unsigned)d.p.N};
    const HaloTma t{bar, d.flag + 1};
    const HaloTma *tma = nullptr;
    if (HALO && tma_halo_fits<TY, TZ>(d.p, e.y, e.z, e.w)) {  // block-uniform
        const bool lead = threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0;
        if (lead) tma_bar_init(bar);
        __syncthreads();
        if (lead)
            tma_load_tile(&tile[0][0][0], &a.phi_map[e.x][cur], e.y * TX - 4, e.z * TY - 1, e.w * TZ - 1, bar,
                          (unsigned)(sizeof(float) * (TZ + 2) * (TY + 2) * HW));
        tma = &t;
    }
    tile_update<float, QG, 15, G_SW, H_SW, true, false, TY, TZ, true, HW>(d.p, lh, lg, d.phi[cur], d.phi[cur ^ 1],
                                                                         d.flag, tile, e.y, e.z, e.w, threadIdx.x,
                                                                         threadIdx.y, threadIdx.z, tma);
}

// One block per entry tiles[blockIdx.x] = (member within the group, bx, by, bz).
template <int QG, bool G_SW, bool H_SW, int TY, int TZ, int HALO>
__global__ void __launch_bounds__(TX *TY *TZ, LBM_MIN_BLOCKS)
    batch_step_kernel(const __grid_constant__ GroupArgs a, const int4 *__restrict__ tiles, int cur, int ntiles) {
    constexpr int HW = HALO ? kTmaRow : TX + 2;
    __shared__ __align__(128) float tile[TZ + 2][TY + 2][HW];
    __shared__ uint64_t bar;
    batch_tile<QG, G_SW, H_SW, TY, TZ, HALO>(a, tiles[blockIdx.x], cur, tile, &bar);
}

// The two-cell step over the table: one block of 16 x 4 x 2 threads per entry
// (member within the group, bx, by, bz) of 32 x 4 x 2 cells.
template <int QG, bool G_SW, bool H_SW>
__global__ void __launch_bounds__(kPairTX *kPairTY *kPairTZ, LBM_PAIR_MIN_BLOCKS)
    batch_pair_kernel(const __grid_constant__ GroupArgs a, const int4 *__restrict__ tiles, int cur) {
    __shared__ __align__(16) float tile[kPairTZ + 2][kPairTY + 2][2 * kPairTX + 4];
    const int4 e = tiles[blockIdx.x];
    const MemberDesc &d = a.m[e.x];
    const pairstep::Lat<float> lh{d.h_rest, d.h_mov, (unsigned)d.p.N}, lg{d.g_rest, d.g_mov, (unsigned)d.p.N};
    pairstep::pair_tile<float, QG, 15, G_SW, H_SW, kPairTX, kPairTY, kPairTZ, true>(
        d.p, lh, lg, d.phi[cur], d.phi[cur ^ 1], d.flag, tile, e.y, e.z, e.w);
}

template <int QG, bool G_SW, bool H_SW, int TY, int TZ>
static cudaError_t launch_shape(int halo, const GroupArgs &a, const int4 *tiles, int ntiles, int cur,
                                cudaStream_t st) {
    if (halo)
        batch_step_kernel<QG, G_SW, H_SW, TY, TZ, 1><<<ntiles, dim3(TX, TY, TZ), 0, st>>>(a, tiles, cur, ntiles);
    else
        batch_step_kernel<QG, G_SW, H_SW, TY, TZ, 0><<<ntiles, dim3(TX, TY, TZ), 0, st>>>(a, tiles, cur, ntiles);
    return cudaGetLastError();
}

template <int QG, bool G_SW, bool H_SW>
static cudaError_t launch_q(int shape, int halo, const GroupArgs &a, const int4 *tiles, int ntiles, int cur,
                            cudaStream_t st) {
    switch (shape) {
        case 0: return launch_shape<QG, G_SW, H_SW, 4, 2>(halo, a, tiles, ntiles, cur, st);
        case 1: return launch_shape<QG, G_SW, H_SW, 8, 1>(halo, a, tiles, ntiles, cur, st);
        case 2: return launch_shape<QG, G_SW, H_SW, 2, 4>(halo, a, tiles, ntiles, cur, st);
        case kPairShape:
            if (halo) return cudaErrorInvalidValue;
            batch_pair_kernel<QG, G_SW, H_SW><<<ntiles, dim3(kPairTX, kPairTY, kPairTZ), 0, st>>>(a, tiles, cur);
            return cudaGetLastError();
        default: return cudaErrorInvalidValue;
    }
}

// g is read swapped on odd time levels; h runs one AA step ahead (opposite layout).
static cudaError_t launch_group(int q_hydro, bool g_sw, int shape, int halo, const GroupArgs &a, const int4 *tiles,
                                int ntiles, int cur, cudaStream_t st) {
    if (ntiles == 0) return cudaSuccess;
    if (q_hydro == 19)
        return g_sw ? launch_q<19, true, false>(shape, halo, a, tiles, ntiles, cur, st)
                    : launch_q<19, false, true>(shape, halo, a, tiles, ntiles, cur, st);
    if (q_hydro == 27)
        return g_sw ? launch_q<27, true, false>(shape, halo, a, tiles, ntiles, cur, st)
                    : launch_q<27, false, true>(shape, halo, a, tiles, ntiles, cur, st);
    return cudaErrorInvalidValue;
}

// cuTensorMapEncodeTiled from the CUDA driver (through the runtime, no link to libcuda)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}

// The tensor map of one phi buffer of an nx x ny x nz box for the TMA halo tile of
// shape (ty, tz); false if the box does not allow it (rows must be a multiple of
// 16 bytes) or the CUDA driver refuses.
bool encode_phi_map(CUtensorMap *m, float *phi, const lbm_domain &d, int ty, int tz) {
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || d.nx % 4 != 0 || ((uintptr_t)phi & 15) != 0) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)d.nx, (cuuint64_t)d.ny, (cuuint64_t)d.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)d.nx * 4, (cuuint64_t)d.nx * d.ny * 4};
    const cuuint32_t box[3] = {(cuuint32_t)kTmaRow, (cuuint32_t)(ty + 2), (cuuint32_t)(tz + 2)};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, phi, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace lbm

struct lbm_batch_t {
    std::vector<lbm_t *> m;
    int q_hydro = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    std::vector<lbm::GroupArgs> groups;  // host copies of the launch parameter blocks
    int4 *d_tiles = nullptr;             // tile table, group after group
    std::vector<int> g_off, g_len;       // each group's range in the table
    int max_tiles = 0;
    int shape = 0, order = 0, table_key = -1;
    int halo = 0;         // phi halo staging: 0 per-thread loads, 1 TMA copy
    bool tma_ok = false;  // every member's phi buffers have tensor maps
    bool pair_ok = false; // every member has nx even: the two-cell tiles apply
    int map_shape = -1;   // the tile shape the tensor maps were encoded for
    cudaGraphExec_t graph[4] = {nullptr, nullptr, nullptr, nullptr};  // key: (t & 1) * 2 + cur
    std::string err;
};

namespace {

lbm_status batch_fail(lbm_batch_t *b, cudaError_t e, const char *what) {
    b->err = std::string(what) + ": " + cudaGetErrorString(e);
    return LBM_ERR_CUDA;
}

#define BATCH_CK(b, call)                                       \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return batch_fail(b, e_, #call); \
    } while (0)

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

struct TileGrid {
    int nbx, nby, nbz;
    int count() const { return nbx * nby * nbz; }
};

TileGrid tile_grid(const lbm_domain &d, int shape) {
    const lbm::TileShape s = lbm::kShapes[shape];
    return {(d.nx + s.tx - 1) / s.tx, (d.ny + s.ty - 1) / s.ty, (d.nz + s.tz - 1) / s.tz};
}

void drop_graphs(lbm_batch_t *b) {
    for (auto &g : b->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

// Fills the tile table for (shape, order).  Order 0 lists each member's tiles
// x fastest, then y, then z, member after member; order 1 deals the members'
// tiles out round robin (member 0 tile 0, member 1 tile 0, ...), so that the
// blocks resident at any moment mix members.
lbm_status build_table(lbm_batch_t *b, int shape, int order) {
    const int key = shape * lbm::kNumOrders + order;
    if (b->table_key == key) return LBM_OK;
    if (b->tma_ok && b->map_shape != shape && shape != lbm::kPairShape) {  // the TMA box is part of the tensor map
        const lbm::TileShape sh = lbm::kShapes[shape];
        for (size_t i = 0; i < b->m.size() && b->tma_ok; ++i) {
            CUtensorMap *maps = b->groups[i / lbm::kGroup].phi_map[i % lbm::kGroup];
            for (int c = 0; c < 2 && b->tma_ok; ++c)
                b->tma_ok = lbm::encode_phi_map(&maps[c], b->m[i]->phi[c], b->m[i]->dom, sh.ty, sh.tz);
        }
        b->map_shape = b->tma_ok ? shape : -1;
        if (!b->tma_ok) b->halo = 0;
    }
    std::vector<int4> t;
    t.reserve(b->max_tiles);
    const int nm = (int)b->m.size();
    b->g_off.clear();
    b->g_len.clear();
    for (int g0 = 0; g0 < nm; g0 += lbm::kGroup) {
        const int g1 = std::min(nm, g0 + lbm::kGroup);
        b->g_off.push_back((int)t.size());
        std::vector<TileGrid> grids;
        int longest = 0;
        for (int i = g0; i < g1; ++i) {
            grids.push_back(tile_grid(b->m[i]->dom, shape));
            longest = std::max(longest, grids.back().count());
        }
        auto entry = [&](int i, int k) {
            const TileGrid &G = grids[i - g0];
            const int bx = k % G.nbx, by = (k / G.nbx) % G.nby, bz = k / (G.nbx * G.nby);
            return make_int4(i - g0, bx, by, bz);
        };
        if (order == 0) {
            for (int i = g0; i < g1; ++i)
                for (int k = 0; k < grids[i - g0].count(); ++k) t.push_back(entry(i, k));
        } else {
            for (int k = 0; k < longest; ++k)
                for (int i = g0; i < g1; ++i)
                    if (k < grids[i - g0].count()) t.push_back(entry(i, k));
        }
        b->g_len.push_back((int)t.size() - b->g_off.back());
    }
    drop_graphs(b);  // captured launches read the table
    BATCH_CK(b, cudaMemcpyAsync(b->d_tiles, t.data(), t.size() * sizeof(int4), cudaMemcpyHostToDevice, b->stream));
    BATCH_CK(b, cudaStreamSynchronize(b->stream));
    b->table_key = key;
    return LBM_OK;
}

// members must be initialised and at the same time level
lbm_status check_lockstep(lbm_batch_t *b) {
    for (lbm_t *s : b->m) {
        if (!s->ready) return b->err = "every member needs a state (lbm_init_phase / lbm_set_state)", LBM_ERR_STATE;
        if (s->t != b->m[0]->t || s->cur != b->m[0]->cur)
            return b->err = "members are at different time levels (stepped outside the batch?)", LBM_ERR_STATE;
    }
    return LBM_OK;
}

// the launches of one time step at level t with phi^t in phi[cur]
cudaError_t enqueue_step(lbm_batch_t *b, int64_t t, int cur) {
    for (size_t g = 0; g < b->groups.size(); ++g) {
        const cudaError_t e = lbm::launch_group(b->q_hydro, (t & 1) != 0, b->shape, b->halo, b->groups[g],
                                                b->d_tiles + b->g_off[g], b->g_len[g], cur, b->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void advance_all(lbm_batch_t *b, int64_t n) {
    for (lbm_t *s : b->m)
        for (int64_t k = 0; k < n; ++k) lbm::advance_level(s);
}

lbm_status graph_for(lbm_batch_t *b, int64_t t, int cur, cudaGraphExec_t *out) {
    const int key = (int)((t & 1) * 2 + cur);
    if (!b->graph[key]) {
        cudaGraph_t g = nullptr;
        BATCH_CK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < lbm::kGraphSteps && e == cudaSuccess; ++k) e = enqueue_step(b, t + k, cur ^ (k & 1));
        const cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return batch_fail(b, e != cudaSuccess ? e : e2, "batch graph capture");
        }
        e = cudaGraphInstantiate(&b->graph[key], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            b->graph[key] = nullptr;
            return batch_fail(b, e, "cudaGraphInstantiate");
        }
    }
    *out = b->graph[key];
    return LBM_OK;
}

struct BatchDeviceGuard {
    int prev = -1;
    bool switched = false;
    explicit BatchDeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) switched = cudaSetDevice(dev) == cudaSuccess;
    }
    ~BatchDeviceGuard() {
        if (switched) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" {

lbm_status lbm_batch_workspace_size(int count, const lbm_domain *doms, const lbm_params *prms, size_t *bytes) {
    if (count < 1 || !doms || !prms || !bytes) return lbm::set_thread_error("count >= 1 and non-NULL arrays"), LBM_ERR_ARG;
    size_t total = 0;
    for (int i = 0; i < count; ++i) {
        size_t b = 0;
        const lbm_status st = lbm_workspace_size(&doms[i], &prms[i], &b);
        if (st != LBM_OK) return st;
        total += align256(b);
    }
    *bytes = total;
    return LBM_OK;
}

lbm_status lbm_batch_create(lbm_batch_t **out, int count, const lbm_domain *doms, const lbm_params *prms,
                            void *cuda_stream, void *workspace, size_t workspace_bytes) {
    if (!out) return lbm::set_thread_error("null output handle"), LBM_ERR_ARG;
    *out = nullptr;
    if (count < 1 || count > 65536 || !doms || !prms)
        return lbm::set_thread_error("a batch has 1..65536 members"), LBM_ERR_ARG;
    for (int i = 0; i < count; ++i) {
        lbm::Params kp;
        std::string why;
        const lbm_status st = lbm::prepare_problem(&doms[i], &prms[i], &kp, &why);
        if (st != LBM_OK) return lbm::set_thread_error("member " + std::to_string(i) + ": " + why), st;
        if (doms[i].q_hydro != doms[0].q_hydro)
            return lbm::set_thread_error("all members need the same hydrodynamic lattice"), LBM_ERR_ARG;
        if (prms[i].precision != LBM_PRECISION_FP32)
            return lbm::set_thread_error("batched stepping supports FP32 storage only"), LBM_ERR_ARG;
        if (prms[i].phase_collision != LBM_PHASE_SRT)
            return lbm::set_thread_error("batched stepping supports the SRT phase collision only"), LBM_ERR_ARG;
        if (prms[i].kernel_form != LBM_FORM_FUSED && prms[i].kernel_form != LBM_FORM_FUSED_CELL)
            return lbm::set_thread_error("batched stepping runs the fused form (one cell per thread) only"),
                   LBM_ERR_ARG;
        if (doms[i].q_phase != 15)
            return lbm::set_thread_error("batched stepping takes the D3Q15 phase-field lattice"), LBM_ERR_ARG;
        if (!lbm::offsets32(kp.N, doms[i].q_hydro, 15))
            return lbm::set_thread_error("member " + std::to_string(i) +
                                         ": (q_hydro - 1) * cells must stay below 2^32 in a batch"),
                   LBM_ERR_ARG;
    }
    if (workspace) {
        size_t need = 0;
        lbm_batch_workspace_size(count, doms, prms, &need);
        if (workspace_bytes < need)
            return lbm::set_thread_error("workspace smaller than lbm_batch_workspace_size()"), LBM_ERR_OOM;
        if (((uintptr_t)workspace & 255) != 0)
            return lbm::set_thread_error("workspace must be 256-byte aligned"), LBM_ERR_ARG;
    }
    lbm_batch_t *b = new (std::nothrow) lbm_batch_t();
    if (!b) return lbm::set_thread_error("out of host memory"), LBM_ERR_OOM;
    b->stream = (cudaStream_t)cuda_stream;
    b->q_hydro = doms[0].q_hydro;
    cudaGetDevice(&b->device);
    char *ws = (char *)workspace;
    for (int i = 0; i < count; ++i) {
        lbm_t *s = nullptr;
        size_t bi = 0;
        lbm_workspace_size(&doms[i], &prms[i], &bi);
        const lbm_status st = lbm_create(&s, &doms[i], &prms[i], cuda_stream, ws, ws ? align256(bi) : 0);
        if (st != LBM_OK) {  // lbm_create has set the thread's error text
            lbm_batch_destroy(b);
            return st;
        }
        b->m.push_back(s);
        if (ws) ws += align256(bi);
    }
    for (int sh = 0; sh < lbm::kNumShapes; ++sh) {
        int n = 0;
        for (lbm_t *s : b->m) n += tile_grid(s->dom, sh).count();
        b->max_tiles = std::max(b->max_tiles, n);
    }
    b->groups.resize((count + lbm::kGroup - 1) / lbm::kGroup);
    for (int i = 0; i < count; ++i) {
        lbm_t *s = b->m[i];
        lbm::MemberDesc &d = b->groups[i / lbm::kGroup].m[i % lbm::kGroup];
        d = lbm::MemberDesc{};
        d.p = s->kp;
        d.h_rest = s->sto.h.rest;
        d.h_mov = static_cast<float *>(s->sto.h.mov);
        d.g_rest = s->sto.g.rest;
        d.g_mov = static_cast<float *>(s->sto.g.mov);
        d.phi[0] = s->phi[0];
        d.phi[1] = s->phi[1];
        d.flag = s->flag;
    }
    b->tma_ok = lbm::tensor_map_encoder() != nullptr;
    b->pair_ok = true;
    for (lbm_t *s : b->m) b->pair_ok = b->pair_ok && s->dom.nx % 2 == 0;
    const cudaError_t e = cudaMalloc(&b->d_tiles, (size_t)b->max_tiles * sizeof(int4));
    if (e != cudaSuccess) {
        lbm::set_thread_error(std::string("batch tile table: ") + cudaGetErrorString(e));
        lbm_batch_destroy(b);
        return LBM_ERR_OOM;
    }
    if (build_table(b, 0, 0) != LBM_OK) {
        lbm::set_thread_error(b->err);
        lbm_batch_destroy(b);
        return LBM_ERR_CUDA;
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_size(const lbm_batch_t *b) { return b ? (int)b->m.size() : 0; }

lbm_t *lbm_batch_member(lbm_batch_t *b, int i) {
    if (!b || i < 0 || i >= (int)b->m.size()) return nullptr;
    return b->m[i];
}

lbm_status lbm_batch_step(lbm_batch_t *b, int64_t n) {
    if (!b || n < 0) return LBM_ERR_ARG;
    BatchDeviceGuard dg(b->device);
    lbm_status st = check_lockstep(b);
    if (st != LBM_OK) return st;
    while (n > 0) {
        const int64_t t = b->m[0]->t;
        const int cur = b->m[0]->cur;
        if (b->stream && n >= lbm::kGraphSteps) {
            cudaGraphExec_t g = nullptr;
            st = graph_for(b, t, cur, &g);
            if (st != LBM_OK) return st;
            BATCH_CK(b, cudaGraphLaunch(g, b->stream));
            advance_all(b, lbm::kGraphSteps);
            n -= lbm::kGraphSteps;
        } else {
            BATCH_CK(b, enqueue_step(b, t, cur));
            advance_all(b, 1);
            n -= 1;
        }
    }
    return LBM_OK;
}

lbm_status lbm_batch_tune(lbm_batch_t *b, int trial_steps, int *choice, double *ms_per_step) {
    if (!b || trial_steps < 1) return LBM_ERR_ARG;
    BatchDeviceGuard dg(b->device);
    lbm_status st = check_lockstep(b);
    if (st != LBM_OK) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BATCH_CK(b, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return b->err = "cudaEventCreate failed", LBM_ERR_CUDA;
    }
    double best = 1e300;
    int best_shape = b->shape, best_order = b->order, best_halo = b->halo;
    for (int ha = 0; ha < lbm::kNumHalos && st == LBM_OK; ++ha) {
        for (int sh = 0; sh < lbm::kNumShapes && st == LBM_OK; ++sh) {
            for (int od = 0; od < lbm::kNumOrders && st == LBM_OK; ++od) {
                const int slot = (ha * lbm::kNumShapes + sh) * lbm::kNumOrders + od;
                if (sh == lbm::kPairShape && (ha == 1 || !b->pair_ok)) {  // two-cell tiles: loads, nx even
                    if (ms_per_step) ms_per_step[slot] = -1.0;
                    continue;
                }
                st = build_table(b, sh, od);
                if (st != LBM_OK) break;
                if (ha == 1 && !b->tma_ok) {  // no tensor maps for these members
                    if (ms_per_step) ms_per_step[slot] = -1.0;
                    continue;
                }
                if (b->halo != ha) drop_graphs(b);
                b->shape = sh;
                b->order = od;
                b->halo = ha;
                cudaError_t e = enqueue_step(b, b->m[0]->t, b->m[0]->cur);  // untimed warm-up step
                advance_all(b, 1);
                if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
                for (int k = 0; k < trial_steps && e == cudaSuccess; ++k) {
                    e = enqueue_step(b, b->m[0]->t, b->m[0]->cur);
                    advance_all(b, 1);
                }
                if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) {
                    st = batch_fail(b, e, "batch tuning");
                    break;
                }
                const double per = ms / trial_steps;
                if (ms_per_step) ms_per_step[slot] = per;
                if (per < best) {
                    best = per;
                    best_shape = sh;
                    best_order = od;
                    best_halo = ha;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LBM_OK) return st;
    st = build_table(b, best_shape, best_order);
    if (st != LBM_OK) return st;
    if (b->halo != best_halo) drop_graphs(b);
    b->shape = best_shape;
    b->order = best_order;
    b->halo = b->tma_ok ? best_halo : 0;
    if (choice) *choice = (b->halo * lbm::kNumShapes + best_shape) * lbm::kNumOrders + best_order;
    return LBM_OK;
}

lbm_status lbm_batch_set_config(lbm_batch_t *b, int choice) {
    if (!b) return LBM_ERR_ARG;
    if (choice < 0 || choice >= lbm::kNumHalos * lbm::kNumShapes * lbm::kNumOrders)
        return b->err = "configuration index out of range", LBM_ERR_ARG;
    const int order = choice % lbm::kNumOrders, shape = (choice / lbm::kNumOrders) % lbm::kNumShapes,
              halo = choice / (lbm::kNumOrders * lbm::kNumShapes);
    BatchDeviceGuard dg(b->device);
    static const char *no_tma =
        "TMA halo staging unavailable (a member's nx is not a multiple of 4, or no driver support)";
    if (halo == 1 && !b->tma_ok) return b->err = no_tma, LBM_ERR_STATE;  // refused before anything changes
    if (shape == lbm::kPairShape && (halo == 1 || !b->pair_ok))
        return b->err = "the two-cell tiles need every member's nx even and per-thread halo loads", LBM_ERR_STATE;
    lbm_status st = build_table(b, shape, order);  // (re)encodes the tensor maps for the shape
    if (st != LBM_OK) return st;
    if (halo == 1 && !b->tma_ok) {
        // the tensor maps of this shape could not be encoded: the table goes back to
        // the configuration in use, so that the next step launches a matching kernel
        st = build_table(b, b->shape, b->order);
        if (st != LBM_OK) return st;
        return b->err = no_tma, LBM_ERR_STATE;
    }
    if (b->halo != halo) drop_graphs(b);
    b->shape = shape;
    b->order = order;
    b->halo = halo;
    return LBM_OK;
}

lbm_status lbm_batch_synchronize(lbm_batch_t *b) {
    if (!b) return LBM_ERR_ARG;
    lbm_status worst = LBM_OK;
    for (size_t i = 0; i < b->m.size(); ++i) {
        const lbm_status st = lbm_synchronize(b->m[i]);
        if (st != LBM_OK && worst == LBM_OK) {
            worst = st;
            b->err = "member " + std::to_string(i) + ": " + lbm_last_error(b->m[i]);
        }
    }
    return worst;
}

const char *lbm_batch_last_error(const lbm_batch_t *b) { return b ? b->err.c_str() : ""; }

void lbm_batch_destroy(lbm_batch_t *b) {
    if (!b) return;
    {
        BatchDeviceGuard dg(b->device);
        if (!b->m.empty()) cudaStreamSynchronize(b->stream);
        drop_graphs(b);
        for (lbm_t *s : b->m) lbm_destroy(s);
        if (b->d_tiles) cudaFree(b->d_tiles);
    }
    delete b;
}

}  // extern "C"
