// lbm_api.cu -- the C ABI declared in include/lbm.h.
//
// Host-side responsibilities: argument validation (before any launch), the
// parameters derived from the problem statement of Section 3 (tau_H, tau_L,
// omega_phi, beta, kappa), the device workspace layout, the time-level and AA
// bookkeeping of Algorithm 2, and host/device transfers.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>

#include "lbm_handle.h"

namespace {

thread_local std::string g_create_error;

struct Layout {
    size_t h_rest, h_mov, g_rest, g_mov, phi0, phi1, flag, red_scratch, red_out, h_tmp, g_tmp, u, total;
};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

size_t storage_bytes(int precision) { return precision == LBM_PRECISION_FP32 ? 4 : 2; }

// rest plane (FP32) then the moving planes in the storage type, for h and g
Layout layout(const lbm_domain &d, int precision, int form) {
    const size_t N = (size_t)d.nx * d.ny * d.nz, b = storage_bytes(precision);
    Layout L;
    size_t off = 0;
    L.h_rest = off;
    off += N * sizeof(float);
    L.h_mov = off;
    off = align256(off + (size_t)(d.q_phase - 1) * N * b);
    L.g_rest = off;
    off += N * sizeof(float);
    L.g_mov = off;
    off = align256(off + (size_t)(d.q_hydro - 1) * N * b);
    L.phi0 = off;
    off = align256(off + N * sizeof(float));
    L.phi1 = off;
    off = align256(off + N * sizeof(float));
    L.flag = off;
    off = align256(off + 256);
    L.red_scratch = off;
    off = align256(off + (size_t)lbm::kReduceBlocks * lbm::kDiagSlots * sizeof(double));
    L.red_out = off;
    off = align256(off + lbm::kDiagSlots * sizeof(double));
    L.h_tmp = L.g_tmp = L.u = 0;
    if (form == LBM_FORM_UNFUSED) {  // second grid of both lattices, stored velocity
        L.h_tmp = off;
        off = align256(off + (size_t)d.q_phase * N * sizeof(float));
        L.g_tmp = off;
        off = align256(off + (size_t)d.q_hydro * N * sizeof(float));
        L.u = off;
        off = align256(off + 3 * N * sizeof(float));
    }
    L.total = off;
    return L;
}

bool finite(double v) { return std::isfinite(v); }

lbm_status validate(const lbm_domain *d, const lbm_params *p, std::string &why) {
    if (!d || !p) return why = "null domain or parameters", LBM_ERR_ARG;
    if (d->nx < 1 || d->ny < 1 || d->nz < 1) return why = "every box size must be >= 1", LBM_ERR_ARG;
    if ((int64_t)d->nx * d->ny * d->nz > (int64_t)INT32_MAX - 1)
        return why = "nx*ny*nz must be < 2^31", LBM_ERR_ARG;
    if (d->nz > 65535 || d->ny > 8 * 65535) return why = "nz must be <= 65535 and ny <= 524280", LBM_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (d->wall[a] != 0 && d->wall[a] != 1) return why = "wall[a] must be 0 (periodic) or 1 (walls)", LBM_ERR_ARG;
    if (d->q_phase != 9 && d->q_phase != 15 && d->q_phase != 19 && d->q_phase != 27)
        return why = "q_phase must be 9, 15, 19 or 27", LBM_ERR_ARG;
    if (d->q_hydro != 9 && d->q_hydro != 19 && d->q_hydro != 27)
        return why = "q_hydro must be 9, 19 or 27", LBM_ERR_ARG;
    if ((d->q_phase == 9) != (d->q_hydro == 9))
        return why = "D2Q9 is a pair: q_phase and q_hydro both 9", LBM_ERR_ARG;
    if (d->q_phase == 9 && (d->nz != 1 || d->wall[2] != 0))
        return why = "the D2Q9 pair needs nz = 1 and no walls on z", LBM_ERR_ARG;
    const double vals[] = {p->rho_H, p->rho_ratio, p->nu_H, p->mu_ratio, p->sigma, p->xi, p->mobility,
                           p->gravity[0], p->gravity[1], p->gravity[2], p->rho_ref};
    for (double v : vals)
        if (!finite(v)) return why = "parameters must be finite", LBM_ERR_ARG;
    if (p->rho_H <= 0 || p->rho_ratio <= 0) return why = "densities must be positive", LBM_ERR_ARG;
    if (p->nu_H <= 0 || p->mu_ratio <= 0) return why = "viscosities must be positive", LBM_ERR_ARG;
    if (p->sigma < 0) return why = "sigma must be >= 0", LBM_ERR_ARG;
    if (p->xi <= 0) return why = "xi must be positive", LBM_ERR_ARG;
    if (p->mobility <= 0) return why = "mobility must be positive", LBM_ERR_ARG;
    if (p->precision != LBM_PRECISION_FP32 && p->precision != LBM_PRECISION_FP16 &&
        p->precision != LBM_PRECISION_BF16)
        return why = "precision must be LBM_PRECISION_FP32, _FP16 or _BF16", LBM_ERR_ARG;
    if (!finite(p->store_phi_ref) || !finite(p->store_g_scale)) return why = "storage parameters must be finite", LBM_ERR_ARG;
    if (p->store_g_scale != 0.0) {
        int ex = 0;
        const double m = std::frexp(p->store_g_scale, &ex);
        if (m != 0.5 || ex < -40 || ex > 40) return why = "store_g_scale must be 0 or a power of two", LBM_ERR_ARG;
    }
    if (p->clamp_phi != 0 && p->clamp_phi != 1) return why = "clamp_phi must be 0 or 1", LBM_ERR_ARG;
    if (p->phase_collision != LBM_PHASE_SRT && p->phase_collision != LBM_PHASE_MRT)
        return why = "phase_collision must be LBM_PHASE_SRT or LBM_PHASE_MRT", LBM_ERR_ARG;
    if (p->phase_collision == LBM_PHASE_MRT && p->precision != LBM_PRECISION_FP32)
        return why = "the MRT phase collision is built for FP32 storage", LBM_ERR_ARG;
    if (p->kernel_form != LBM_FORM_FUSED && p->kernel_form != LBM_FORM_UNFUSED &&
        p->kernel_form != LBM_FORM_FUSED_CELL && p->kernel_form != LBM_FORM_FUSED_PAIR)
        return why = "kernel_form must be LBM_FORM_FUSED, _UNFUSED, _FUSED_CELL or _FUSED_PAIR", LBM_ERR_ARG;
    if (p->kernel_form == LBM_FORM_UNFUSED && p->precision != LBM_PRECISION_FP32)
        return why = "the unfused form is built for FP32 storage", LBM_ERR_ARG;
    if (p->kernel_form == LBM_FORM_FUSED_PAIR && d->nx % 2 != 0)
        return why = "the two-cell fused step needs nx even", LBM_ERR_ARG;
    if (d->q_phase != 15 && (p->precision != LBM_PRECISION_FP32 || p->phase_collision != LBM_PHASE_SRT ||
                             p->kernel_form == LBM_FORM_UNFUSED))
        return why = "the D2Q9 / D3Q19 / D3Q27 phase lattices run with FP32 storage, SRT, fused form", LBM_ERR_ARG;
    if (d->q_phase == 9 && p->gravity[2] != 0.0)
        return why = "the D2Q9 pair carries no z momentum: gravity[2] must be 0", LBM_ERR_ARG;
    if (!lbm::offsets32((long long)d->nx * d->ny * d->nz, d->q_hydro, d->q_phase) &&
        (p->precision != LBM_PRECISION_FP32 || d->q_phase != 15))
        return why = "boxes with (q - 1) nx ny nz >= 2^32 run with FP32 storage and the D3Q15 phase lattice",
               LBM_ERR_ARG;
    const double rho_L = p->rho_H / p->rho_ratio;
    const double nu_L = p->nu_H * p->rho_H / (p->mu_ratio * rho_L);
    if (!(rho_L > 0) || !finite(rho_L)) return why = "rho_L = rho_H / rho_ratio must be positive", LBM_ERR_ARG;
    if (!(nu_L > 0) || !finite(nu_L)) return why = "nu_L must be positive", LBM_ERR_ARG;
    return LBM_OK;
}

// Section 3: nu = tau c_s^2, M = tau_phi c_s^2, s_nu = 1/(tau + 1/2),
// omega_phi = 1/(tau_phi + 1/2), beta = 12 sigma/xi, kappa = 3 sigma xi/2.
lbm::Params derive(const lbm_domain &d, const lbm_params &p) {
    lbm::Params k;
    k.nx = d.nx;
    k.ny = d.ny;
    k.nz = d.nz;
    k.wall = (d.wall[0] ? 1 : 0) | (d.wall[1] ? 2 : 0) | (d.wall[2] ? 4 : 0);
    k.N = (long long)d.nx * d.ny * d.nz;
    const double cs2 = 1.0 / 3.0;
    const double rho_L = p.rho_H / p.rho_ratio;
    const double nu_L = p.nu_H * p.rho_H / (p.mu_ratio * rho_L);
    const double tau_H = p.nu_H / cs2, tau_L = nu_L / cs2;
    k.rho_L = (float)rho_L;
    k.drho = (float)(p.rho_H - rho_L);
    k.tau_L = (float)tau_L;
    k.dtau = (float)(tau_H - tau_L);
    k.omega_phi = (float)(1.0 / (p.mobility / cs2 + 0.5));
    k.beta4 = (float)(4.0 * 12.0 * p.sigma / p.xi);
    k.kappa = (float)(1.5 * p.sigma * p.xi);
    k.inv_xi = (float)(1.0 / p.xi);
    k.gx = (float)p.gravity[0];
    k.gy = (float)p.gravity[1];
    k.gz = (float)p.gravity[2];
    k.rho_ref = (float)p.rho_ref;
    k.phi_lo = p.clamp_phi ? 0.0f : -INFINITY;
    k.phi_hi = p.clamp_phi ? 1.0f : INFINITY;
    k.phase_mrt = p.phase_collision == LBM_PHASE_MRT ? 1 : 0;
    k.step_form = p.kernel_form == LBM_FORM_FUSED_CELL || p.kernel_form == LBM_FORM_FUSED_PAIR ? p.kernel_form : 0;
    if (p.precision == LBM_PRECISION_FP32) {
        k.h_ref = 0.0f;
        k.g_scale = k.g_inv_scale = 1.0f;
    } else {
        const double gs = p.store_g_scale != 0.0 ? p.store_g_scale : (p.precision == LBM_PRECISION_FP16 ? 4096.0 : 1.0);
        k.h_ref = (float)p.store_phi_ref;
        k.g_scale = (float)gs;
        k.g_inv_scale = (float)(1.0 / gs);
    }
    return k;
}

struct DeviceGuard {
    int prev = -1;
    bool switched = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) switched = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (switched) cudaSetDevice(prev);
    }
};

lbm_status cuda_fail(lbm_t *s, cudaError_t e, const char *what) {
    s->err = std::string(what) + ": " + cudaGetErrorString(e);
    return LBM_ERR_CUDA;
}

#define LBM_CK(s, call)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(s, e_, #call); \
    } while (0)

// In-place AA layout of each lattice at the current level (the unfused form
// keeps both natural).
bool g_swapped(const lbm_t *s) { return !s->unfused && (s->t & 1) != 0; }
bool h_swapped(const lbm_t *s) { return !s->unfused && ((s->t + 1) & 1) != 0; }
size_t plane_bytes(const lbm_t *s) { return (size_t)s->kp.N * sizeof(float); }

cudaMemcpyKind kind_to_device(int on_device) { return on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }

// One time step's launch(es) at the handle's current level.
cudaError_t enqueue_one(lbm_t *s) {
    if (s->unfused)
        return lbm::launch_unfused(s->kp, s->uf, s->sto, s->dom.q_hydro, true, s->phi[s->cur], s->phi[s->cur ^ 1],
                                   s->flag, s->stream);
    return lbm::launch_step(s->kp, s->sto, s->dom.q_hydro, s->dom.q_phase, g_swapped(s), h_swapped(s), true,
                            s->phi[s->cur], s->phi[s->cur ^ 1], s->flag, s->stream);
}

// Small boxes spend most of a step launching it: runs of kStepGraph steps are
// replayed from a CUDA graph (captured on first use, one per starting parity and
// phi buffer) when the handle has its own stream that nobody is capturing.
constexpr int kStepGraph = 16;
constexpr long long kStepGraphCells = 1ll << 23;  // boxes up to 8 M cells

lbm_status step_graph_for(lbm_t *s, cudaGraphExec_t *out) {
    const int key = (int)((s->t & 1) * 2 + s->cur);
    if (!s->step_graph[key]) {
        const int64_t t0 = s->t;
        const int c0 = s->cur;
        cudaGraph_t g = nullptr;
        LBM_CK(s, cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < kStepGraph && e == cudaSuccess; ++k) {
            e = enqueue_one(s);
            s->cur ^= 1;
            s->t += 1;
        }
        s->t = t0;  // capture enqueues nothing: the level stays until the graph runs
        s->cur = c0;
        const cudaError_t e2 = cudaStreamEndCapture(s->stream, &g);
        if (e == cudaSuccess && e2 == cudaSuccess) e = cudaGraphInstantiate(&s->step_graph[key], g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            s->step_graph[key] = nullptr;
            return cuda_fail(s, e != cudaSuccess ? e : e2, "step graph capture");
        }
    }
    *out = s->step_graph[key];
    return LBM_OK;
}

bool step_graphs_apply(const lbm_t *s) {
    if (!s->stream || s->kp.N > kStepGraphCells) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s->stream, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
}

void drop_step_graphs(lbm_t *s) {
    for (auto &g : s->step_graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

}  // namespace

namespace lbm {
// Validation and derived parameters for entry points outside this file.
lbm_status prepare_problem(const lbm_domain *dom, const lbm_params *prm, Params *out, std::string *why) {
    std::string w;
    const lbm_status st = validate(dom, prm, w);
    if (st != LBM_OK) {
        if (why) *why = w;
        return st;
    }
    *out = derive(*dom, *prm);
    return LBM_OK;
}

// Message returned by lbm_last_error(NULL) for a call without a handle.
void set_thread_error(const std::string &msg) { g_create_error = msg; }
}  // namespace lbm

extern "C" {

lbm_status lbm_workspace_size(const lbm_domain *dom, const lbm_params *prm, size_t *bytes) {
    std::string why;
    if (!bytes) return LBM_ERR_ARG;
    lbm_status st = validate(dom, prm, why);
    if (st != LBM_OK) {
        g_create_error = why;
        return st;
    }
    *bytes = layout(*dom, prm->precision, prm->kernel_form).total;
    return LBM_OK;
}

lbm_status lbm_create(lbm_t **out, const lbm_domain *dom, const lbm_params *prm, void *cuda_stream, void *workspace,
                      size_t workspace_bytes) {
    if (!out) return g_create_error = "null output handle", LBM_ERR_ARG;
    *out = nullptr;
    std::string why;
    lbm_status st = validate(dom, prm, why);
    if (st != LBM_OK) return g_create_error = why, st;
    const Layout L = layout(*dom, prm->precision, prm->kernel_form);
    if (workspace) {
        if (workspace_bytes < L.total) return g_create_error = "workspace smaller than lbm_workspace_size()", LBM_ERR_OOM;
        if (((uintptr_t)workspace & 255) != 0) return g_create_error = "workspace must be 256-byte aligned", LBM_ERR_ARG;
    }
    lbm_t *s = new (std::nothrow) lbm_t();
    if (!s) return g_create_error = "host allocation failed", LBM_ERR_OOM;
    s->dom = *dom;
    s->prm = *prm;
    s->kp = derive(*dom, *prm);
    s->stream = (cudaStream_t)cuda_stream;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        g_create_error = "no CUDA device";
        delete s;
        return LBM_ERR_CUDA;
    }
    if (workspace) {
        s->ws = (char *)workspace;
        s->owns_ws = false;
    } else {
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, L.total);
        if (e != cudaSuccess) {
            g_create_error = std::string("cudaMalloc of the workspace failed: ") + cudaGetErrorString(e);
            cudaGetLastError();
            delete s;
            return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
        }
        s->ws = (char *)p;
        s->owns_ws = true;
    }
    s->ws_bytes = L.total;
    s->sto.precision = prm->precision;
    s->sto.h.rest = (float *)(s->ws + L.h_rest);
    s->sto.h.mov = s->ws + L.h_mov;
    s->sto.g.rest = (float *)(s->ws + L.g_rest);
    s->sto.g.mov = s->ws + L.g_mov;
    s->phi[0] = (float *)(s->ws + L.phi0);
    s->phi[1] = (float *)(s->ws + L.phi1);
    s->flag = (int *)(s->ws + L.flag);
    s->red_scratch = (double *)(s->ws + L.red_scratch);
    s->red_out = (double *)(s->ws + L.red_out);
    s->unfused = prm->kernel_form == LBM_FORM_UNFUSED;
    s->uf.h_tmp = s->unfused ? (float *)(s->ws + L.h_tmp) : nullptr;
    s->uf.g_tmp = s->unfused ? (float *)(s->ws + L.g_tmp) : nullptr;
    s->uf.u = s->unfused ? (float *)(s->ws + L.u) : nullptr;
    s->cur = 0;
    s->t = 0;
    s->ready = false;
    cudaError_t e = cudaMemsetAsync(s->flag, 0, 2 * sizeof(int), s->stream);
    if (e != cudaSuccess) {
        g_create_error = std::string("cudaMemsetAsync: ") + cudaGetErrorString(e);
        if (s->owns_ws) cudaFree(s->ws);
        delete s;
        return LBM_ERR_CUDA;
    }
    *out = s;
    return LBM_OK;
}

lbm_status lbm_init_phase(lbm_t *s, const float *phi0, int phi0_on_device) {
    if (!s || !phi0) return LBM_ERR_ARG;
    DeviceGuard dg(s->device);
    LBM_CK(s, cudaMemcpyAsync(s->phi[0], phi0, plane_bytes(s), kind_to_device(phi0_on_device), s->stream));
    if (!phi0_on_device) LBM_CK(s, cudaStreamSynchronize(s->stream));
    LBM_CK(s, lbm::launch_init(s->kp, s->sto, s->dom.q_hydro, s->dom.q_phase, s->phi[0], s->stream));
    LBM_CK(s, cudaMemsetAsync(s->flag, 0, 2 * sizeof(int), s->stream));
    // time level 0: the first phase-field step alone (u_{-1} = 0, phi^{-1} = phi0)
    if (s->unfused) {
        LBM_CK(s, cudaMemsetAsync(s->uf.u, 0, 3 * plane_bytes(s), s->stream));
        LBM_CK(s, lbm::launch_unfused(s->kp, s->uf, s->sto, s->dom.q_hydro, false, s->phi[0], s->phi[1], s->flag,
                                      s->stream));
    } else {
        LBM_CK(s, lbm::launch_step(s->kp, s->sto, s->dom.q_hydro, s->dom.q_phase, false, false, false, s->phi[0], s->phi[1],
                                   s->flag, s->stream));
    }
    s->cur = 1;
    s->t = 0;
    s->ready = true;
    return LBM_OK;
}

lbm_status lbm_step(lbm_t *s, int64_t n) {
    if (!s || n < 0) return LBM_ERR_ARG;
    if (!s->ready) return s->err = "lbm_step before lbm_init_phase / lbm_set_state", LBM_ERR_STATE;
    DeviceGuard dg(s->device);
    const bool graphs = n >= kStepGraph && step_graphs_apply(s);
    while (n > 0) {
        if (graphs && n >= kStepGraph) {
            cudaGraphExec_t g = nullptr;
            const lbm_status st = step_graph_for(s, &g);
            if (st != LBM_OK) return st;
            LBM_CK(s, cudaGraphLaunch(g, s->stream));
            s->cur ^= kStepGraph & 1;
            s->t += kStepGraph;
            n -= kStepGraph;
        } else {
            LBM_CK(s, enqueue_one(s));
            s->cur ^= 1;
            s->t += 1;
            n -= 1;
        }
    }
    return LBM_OK;
}

lbm_status lbm_get_fields(lbm_t *s, float *phi, float *u, float *p, int on_device) {
    if (!s) return LBM_ERR_ARG;
    if (!s->ready) return s->err = "no state yet", LBM_ERR_STATE;
    DeviceGuard dg(s->device);
    const size_t N = (size_t)s->kp.N;
    const float *cur = s->phi[s->cur];
    if (on_device) {
        LBM_CK(s, lbm::launch_fields(s->kp, s->sto, s->dom.q_hydro, g_swapped(s), cur, phi, u ? u : nullptr,
                                     u ? u + N : nullptr, u ? u + 2 * N : nullptr, p, s->stream));
        return LBM_OK;
    }
    // host outputs: one plane at a time through the idle phi buffer
    float *stage = s->phi[s->cur ^ 1];
    if (phi) LBM_CK(s, cudaMemcpyAsync(phi, cur, plane_bytes(s), cudaMemcpyDeviceToHost, s->stream));
    for (int comp = 0; comp < 4; ++comp) {
        float *dst = comp < 3 ? (u ? u + comp * N : nullptr) : p;
        if (!dst) continue;
        LBM_CK(s, lbm::launch_fields(s->kp, s->sto, s->dom.q_hydro, g_swapped(s), cur, nullptr,
                                     comp == 0 ? stage : nullptr, comp == 1 ? stage : nullptr,
                                     comp == 2 ? stage : nullptr, comp == 3 ? stage : nullptr, s->stream));
        LBM_CK(s, cudaMemcpyAsync(dst, stage, plane_bytes(s), cudaMemcpyDeviceToHost, s->stream));
    }
    LBM_CK(s, cudaStreamSynchronize(s->stream));
    return LBM_OK;
}

lbm_status lbm_reduce(lbm_t *s, double *out) {
    if (!s || !out) return LBM_ERR_ARG;
    if (!s->ready) return s->err = "no state yet", LBM_ERR_STATE;
    DeviceGuard dg(s->device);
    LBM_CK(s, lbm::launch_reduce(s->kp, s->sto, s->dom.q_hydro, g_swapped(s), s->phi[s->cur], s->red_scratch,
                                 s->red_out, s->stream));
    double raw[LBM_DIAG_COUNT];
    LBM_CK(s, cudaMemcpyAsync(raw, s->red_out, sizeof(raw), cudaMemcpyDeviceToHost, s->stream));
    LBM_CK(s, cudaStreamSynchronize(s->stream));
    const double V = raw[LBM_DIAG_LIGHT_VOL];
    for (int k = 0; k < LBM_DIAG_COUNT; ++k) out[k] = raw[k];
    for (int k = LBM_DIAG_LIGHT_X; k <= LBM_DIAG_LIGHT_UZ; ++k) out[k] = V != 0.0 ? raw[k] / V : 0.0;
    return LBM_OK;
}

lbm_status lbm_get_state(lbm_t *s, float *h, float *g, float *phi, int on_device) {
    if (!s) return LBM_ERR_ARG;
    if (!s->ready) return s->err = "no state yet", LBM_ERR_STATE;
    DeviceGuard dg(s->device);
    const size_t N = (size_t)s->kp.N;
    const int Q = s->dom.q_hydro;
    if (on_device) {
        if (h) LBM_CK(s, lbm::launch_gather(s->kp, s->sto, true, s->dom.q_phase, h_swapped(s), 0, s->dom.q_phase, h, s->stream));
        if (g) LBM_CK(s, lbm::launch_gather(s->kp, s->sto, false, Q, g_swapped(s), 0, Q, g, s->stream));
        if (phi) LBM_CK(s, cudaMemcpyAsync(phi, s->phi[s->cur], plane_bytes(s), cudaMemcpyDeviceToDevice, s->stream));
        return LBM_OK;
    }
    float *stage = s->phi[s->cur ^ 1];
    for (int i = 0; h && i < s->dom.q_phase; ++i) {
        LBM_CK(s, lbm::launch_gather(s->kp, s->sto, true, s->dom.q_phase, h_swapped(s), i, i + 1, stage, s->stream));
        LBM_CK(s, cudaMemcpyAsync(h + i * N, stage, plane_bytes(s), cudaMemcpyDeviceToHost, s->stream));
    }
    for (int i = 0; g && i < Q; ++i) {
        LBM_CK(s, lbm::launch_gather(s->kp, s->sto, false, Q, g_swapped(s), i, i + 1, stage, s->stream));
        LBM_CK(s, cudaMemcpyAsync(g + i * N, stage, plane_bytes(s), cudaMemcpyDeviceToHost, s->stream));
    }
    if (phi) LBM_CK(s, cudaMemcpyAsync(phi, s->phi[s->cur], plane_bytes(s), cudaMemcpyDeviceToHost, s->stream));
    LBM_CK(s, cudaStreamSynchronize(s->stream));
    return LBM_OK;
}

lbm_status lbm_set_state(lbm_t *s, const float *h, const float *g, const float *phi, int on_device) {
    if (!s || !h || !g || !phi) return LBM_ERR_ARG;
    DeviceGuard dg(s->device);
    const size_t N = (size_t)s->kp.N;
    const int Q = s->dom.q_hydro;
    // the state becomes time level 0: g natural, h one AA step ahead (swapped)
    s->t = 0;
    if (on_device) {
        LBM_CK(s, lbm::launch_scatter(s->kp, s->sto, true, s->dom.q_phase, h_swapped(s), 0, s->dom.q_phase, h, s->stream));
        LBM_CK(s, lbm::launch_scatter(s->kp, s->sto, false, Q, g_swapped(s), 0, Q, g, s->stream));
        LBM_CK(s, cudaMemcpyAsync(s->phi[s->cur], phi, plane_bytes(s), cudaMemcpyDeviceToDevice, s->stream));
    } else {
        float *stage = s->phi[s->cur ^ 1];
        for (int i = 0; i < s->dom.q_phase; ++i) {
            LBM_CK(s, cudaMemcpyAsync(stage, h + i * N, plane_bytes(s), cudaMemcpyHostToDevice, s->stream));
            LBM_CK(s, lbm::launch_scatter(s->kp, s->sto, true, s->dom.q_phase, h_swapped(s), i, i + 1, stage, s->stream));
        }
        for (int i = 0; i < Q; ++i) {
            LBM_CK(s, cudaMemcpyAsync(stage, g + i * N, plane_bytes(s), cudaMemcpyHostToDevice, s->stream));
            LBM_CK(s, lbm::launch_scatter(s->kp, s->sto, false, Q, g_swapped(s), i, i + 1, stage, s->stream));
        }
        LBM_CK(s, cudaMemcpyAsync(s->phi[s->cur], phi, plane_bytes(s), cudaMemcpyHostToDevice, s->stream));
        LBM_CK(s, cudaStreamSynchronize(s->stream));
    }
    LBM_CK(s, cudaMemsetAsync(s->flag, 0, 2 * sizeof(int), s->stream));
    s->ready = true;
    return LBM_OK;
}

lbm_status lbm_synchronize(lbm_t *s) {
    if (!s) return LBM_ERR_ARG;
    DeviceGuard dg(s->device);
    int flag[2] = {0, 0};  // [0] divergence, [1] a TMA copy of the phi tile that did not complete (batch)
    LBM_CK(s, cudaMemcpyAsync(flag, s->flag, sizeof(flag), cudaMemcpyDeviceToHost, s->stream));
    LBM_CK(s, cudaStreamSynchronize(s->stream));
    if (flag[1]) return s->err = "a TMA copy of the phi halo tile did not complete on the device", LBM_ERR_CUDA;
    if (flag[0]) return s->err = "non-finite phi or p* produced on the device", LBM_ERR_DIVERGED;
    return LBM_OK;
}

int64_t lbm_steps_done(const lbm_t *s) { return s ? s->t : -1; }

const char *lbm_last_error(const lbm_t *s) { return s ? s->err.c_str() : g_create_error.c_str(); }

void lbm_destroy(lbm_t *s) {
    if (!s) return;
    {
        DeviceGuard dg(s->device);
        cudaStreamSynchronize(s->stream);
        drop_step_graphs(s);
        if (s->owns_ws) cudaFree(s->ws);
    }
    delete s;
}

}  // extern "C"
