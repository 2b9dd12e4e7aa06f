/*
 * lbm.h -- C ABI of the GB300 (sm_103a) conservative Allen-Cahn multiphase
 * lattice Boltzmann solver.
 *
 * Method: Holzer, Bauer, Koestler, Ruede, "Highly efficient lattice Boltzmann
 * multiphase simulations of immiscible fluids at high-density ratios on CPUs and
 * GPUs through code generation", arXiv 2012.06144.
 *   - phase-field LB on D3Q15, or D3Q19 / D3Q27 (and the D2Q9 pair in two
 *     dimensions) for the other stencil pairs of Section 5.1 (Section 3.1,
 *     eq:lb_interface, eq:interfaceTracking,
 *     eq:updatePhaseField), single-relaxation-time collision with rate
 *     omega_phi = 1/(3 M + 1/2);
 *   - velocity-based hydrodynamic LB on D3Q19 or D3Q27 (D2Q9 in the pair) (Section 3.2, eq:lb_flow,
 *     eq:forceHydro ... eq:updateVelocityField), weighted-orthogonal MRT with the
 *     force applied in moment space (eq:improved_collision);
 *   - isotropic stencils eq:grad and eq:lap;
 *   - one coupled time step = phase step then hydro step (Algorithm 2).
 *
 * Conventions shared by every entry point
 *   - Cells: index c = x + nx*(y + ny*z), x fastest.  Scalar fields are nx*ny*nz
 *     floats; vector fields are three such planes (x, y, z components).
 *   - Populations: structure of arrays, plane i holds direction i for all cells.
 *     Direction numbering (both lattices): 0 = rest; 1..6 = +x,-x,+y,-y,+z,-z;
 *     D3Q19/D3Q27 then 7..18 = edges (+x+y,-x-y,+x-y,-x+y, +x+z,-x-z,+x-z,-x+z,
 *     +y+z,-y-z,+y-z,-y+z); D3Q27 then 19..26 = corners (+++,---,++-,--+,+-+,-+-,
 *     -++,+--).  D3Q15 = rest, the six faces, then the eight corners as 7..14 in
 *     the same corner order.  D2Q9 = rest, +x,-x,+y,-y, then the xy edges
 *     +x+y,-x-y,+x-y,-x+y as 5..8.  Each moving direction is followed by its
 *     opposite.
 *   - Walls: wall[a] = 1 puts no-slip walls (half-way bounce-back for h and g,
 *     mirrored ghost values of phi in the stencils) on both faces of axis a;
 *     wall[a] = 0 makes axis a periodic.
 *   - Pointers flagged "on_device" are device pointers (any CUDA allocation
 *     visible to the library's device); otherwise they are host pointers.  The
 *     caller owns every buffer it passes; the library never frees or retains
 *     them beyond the call.
 *   - Every call is enqueued on the stream given to lbm_create.  Calls that
 *     return data to host memory synchronise that stream before returning.
 *   - No call aborts, exits or traps.  Invalid arguments return LBM_ERR_ARG
 *     before anything is launched; CUDA failures return LBM_ERR_CUDA; the text
 *     of the last failure is available from lbm_last_error.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_t lbm_t; /* opaque simulation handle */

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = -1,      /* invalid argument or parameter                       */
    LBM_ERR_CUDA = -2,     /* a CUDA runtime call or kernel launch failed          */
    LBM_ERR_OOM = -3,      /* workspace too small or allocation failed             */
    LBM_ERR_DIVERGED = -4, /* a non-finite phi or p* was produced on the device    */
    LBM_ERR_STATE = -5     /* call out of order (e.g. lbm_step before initialising) */
} lbm_status;

/* Storage of the populations in device memory.  Arithmetic is FP32 in every case.
 * FP32: every population in FP32.  FP16 / BF16: the rest populations h_0, g_0
 * stay FP32 and the moving ones are stored in 16 bits as shifted, scaled
 * deviations: h_i as h_i - w_i * store_phi_ref, g_i as g_i * store_g_scale.  The
 * rest population absorbs the rounding of the others, so the phase mass sum phi
 * and the hydrodynamic p* are kept to FP32 rounding. */
enum { LBM_PRECISION_FP32 = 0, LBM_PRECISION_FP16 = 1, LBM_PRECISION_BF16 = 2 };

/* Phase-field collision.  SRT: Omega = omega_phi I (Section 5's D3Q15 SRT, the
 * benchmarked form).  MRT: Omega = M^-1 S M of Section 3.1 with the first-order
 * moments relaxed by omega_phi and all other moments by 1, in a moment basis
 * orthogonal under the lattice weights; computed in closed form as
 * h*_i = h^eq_i + F_i/2 + (1 - omega_phi) w_i e_i . J / c_s^2 with
 * J = sum_j e_j (h_j - h^eq_j + F_j/2).  MRT needs FP32 storage and a single
 * simulation (not a batch member). */
enum { LBM_PHASE_SRT = 0, LBM_PHASE_MRT = 1 };

/* Kernel form of a time step.  FUSED: one kernel per step (Algorithm 2 with the
 * hydro(k-1) + phase(k) bracketing, in-place AA streaming, one copy of each
 * lattice: 344 B moved per cell at D3Q27), in the variant the library measured
 * faster: FUSED_PAIR wherever it applies, for every storage format, FUSED_CELL
 * otherwise.  UNFUSED: the passes of the paper's straightforward
 * Algorithm 1 -- a collision kernel for each lattice (storing u and phi) and a
 * streaming kernel for each, over two grids (708 B per cell at D3Q27) --
 * computing the same update; the baseline the fused form is measured against
 * (Section 4.2).  UNFUSED needs FP32 storage and a single simulation.
 * FUSED_CELL: the fused step with one cell per thread.  FUSED_PAIR: the fused
 * step with two neighbouring cells (x, x + 1) per thread, their arithmetic in
 * packed FP32 pairs and their population pairs moved by one access where they
 * are neighbours in memory; needs nx even, and takes every lattice pair, phase
 * collision and box size that the problem allows otherwise.  All fused variants
 * compute
 * the same update; they differ in rounding only where a multiply and an add
 * are fused differently. */
enum { LBM_FORM_FUSED = 0, LBM_FORM_UNFUSED = 1, LBM_FORM_FUSED_CELL = 2, LBM_FORM_FUSED_PAIR = 3 };

/* Box and lattices (Section 3; Section 5 uses D3Q15 for h and D3Q27 for g). */
typedef struct {
    int nx, ny, nz; /* cells per axis, each >= 1, nx*ny*nz < 2^31,
                       ny <= 524280, nz <= 65535 (launch-grid limits); boxes
                       with (max(q_phase, q_hydro) - 1) nx ny nz >= 2^32 (about
                       165 M cells at D3Q27) need FP32 storage and the D3Q15
                       phase lattice                                           */
    int wall[3];    /* 0 = periodic axis, 1 = no-slip walls on both faces       */
    int q_phase;    /* 15 (the benchmarked pair), 19 or 27; or 9 with q_hydro 9
                       (the two-dimensional D2Q9 pair of Section 5.1: nz = 1,
                       wall[2] = 0, gravity[2] = 0).  9, 19 and 27 need FP32
                       storage, the SRT phase collision and the fused form      */
    int q_hydro;    /* 19 or 27; 9 only with q_phase 9                          */
} lbm_domain;

/* Physical parameters in lattice units (Delta x = Delta t = 1, c_s^2 = 1/3). */
typedef struct {
    double rho_H;      /* heavy-fluid density (phi = 1), > 0                    */
    double rho_ratio;  /* rho_H / rho_L, > 0                 (eq:density)       */
    double nu_H;       /* heavy-fluid kinematic viscosity, > 0                  */
    double mu_ratio;   /* mu_H / mu_L with mu = rho nu, > 0                      */
    double sigma;      /* surface tension, >= 0: beta = 12 sigma/xi, kappa = 3 sigma xi/2 (eq:chemPot) */
    double xi;         /* interface width, > 0                                   */
    double mobility;   /* M = tau_phi c_s^2, > 0              (eq:mobility)      */
    double gravity[3]; /* body-force acceleration g                              */
    double rho_ref;    /* buoyancy F_b = (rho - rho_ref) g; rho_ref = 0 gives F_b = rho g */
    int precision;     /* LBM_PRECISION_FP32, _FP16 or _BF16 (population storage)  */
    int clamp_phi;     /* 1: use phi clamped to [0, 1] inside rho and tau (keeps
                          rho >= rho_L when phi undershoots at high density ratio);
                          0: use phi as is                                       */
    double store_phi_ref; /* 16-bit storage: shift of h (1 suits boxes that are mostly
                             heavy fluid, 0 mostly light); ignored for FP32          */
    double store_g_scale; /* 16-bit storage: power of two scaling g into the format's
                             normal range; 0 selects 4096 (FP16) or 1 (BF16)        */
    int phase_collision;  /* LBM_PHASE_SRT or LBM_PHASE_MRT                          */
    int kernel_form;      /* LBM_FORM_FUSED, _UNFUSED, _FUSED_CELL or _FUSED_PAIR      */
} lbm_params;

/* Diagnostics returned by lbm_reduce (FP64 accumulation).  "Light" weights a
 * cell by the bubble indicator b = clamp(1 - 2 phi, 0, 1): 1 in the light phase,
 * falling to 0 at the interface's mid-level phi = 1/2 and 0 beyond, so that the
 * heavy bulk -- where acoustic waves move phi by ~1e-4 around 1 over millions
 * of cells -- does not enter the bubble's centroid and velocity. */
enum {
    LBM_DIAG_MASS = 0,    /* sum phi                                               */
    LBM_DIAG_MOM_X = 1,   /* sum rho u_x   (rho from eq:density, phi clamped if clamp_phi) */
    LBM_DIAG_MOM_Y = 2,
    LBM_DIAG_MOM_Z = 3,
    LBM_DIAG_LIGHT_VOL = 4,  /* sum b                                              */
    LBM_DIAG_LIGHT_X = 5,    /* sum (x + 1/2) b / sum b: centroid                  */
    LBM_DIAG_LIGHT_Y = 6,
    LBM_DIAG_LIGHT_Z = 7,
    LBM_DIAG_LIGHT_UX = 8,   /* sum u_x b / sum b: rise velocity                   */
    LBM_DIAG_LIGHT_UY = 9,
    LBM_DIAG_LIGHT_UZ = 10,
    LBM_DIAG_MAX_U = 11,     /* max |u|                                            */
    LBM_DIAG_COUNT = 12
};

/* Bytes of device workspace lbm_create needs for this problem (populations h
 * and g, two phi buffers, flags and reduction scratch; the unfused form adds a
 * second grid of both lattices and the velocity field).  Host-only; never
 * touches the GPU. */
lbm_status lbm_workspace_size(const lbm_domain *dom, const lbm_params *prm, size_t *bytes);

/* Validates the problem (Section 3 parameters; LBM_ERR_ARG on a non-positive
 * size, q_phase not 9/15/19/27, q_hydro not 9/19/27, a D2Q9 lattice not paired with
 * D2Q9 or on a box that is not nx x ny x 1 periodic in z, non-positive densities, viscosities,
 * xi or mobility, negative sigma, non-finite values), derives tau_H, tau_L,
 * omega_phi, beta, kappa and creates a handle on the current CUDA device.
 * cuda_stream: a cudaStream_t to enqueue all work on, or NULL for the legacy
 * default stream.  workspace: a device buffer of at least lbm_workspace_size()
 * bytes, 256-byte aligned, owned by the caller and kept alive until
 * lbm_destroy; or NULL to let the library allocate (and later free) it. */
lbm_status lbm_create(lbm_t **out, const lbm_domain *dom, const lbm_params *prm, void *cuda_stream,
                      void *workspace, size_t workspace_bytes);

/* Initial state from a phase field phi0 (nx*ny*nz floats): h_i = w_i phi0
 * (= phi0 Gamma_i at rest), g_i = 0 (p* = 0, u = 0).  Runs the first phase-field
 * step so that the handle holds time level 0.  Resets the step counter. */
lbm_status lbm_init_phase(lbm_t *s, const float *phi0, int phi0_on_device);

/* Advances n >= 0 coupled time steps (Algorithm 2: phase step, hydro step).
 * Asynchronous: returns after enqueueing.  On a stream of its own (not NULL) and
 * for boxes of at most 8,388,608 cells, runs of 16 steps are replayed from CUDA
 * graphs captured on first use (one per starting AA parity and phi buffer, kept
 * until lbm_destroy), so the first call with n >= 16 takes longer; while the
 * stream is being captured by the caller, every step is launched directly. */
lbm_status lbm_step(lbm_t *s, int64_t n);

/* Macroscopic fields at the current time level t: phi = sum_i h_i
 * (eq:updatePhaseField), u = sum_i g_i e_i + F/(2 rho) (eq:updateVelocityField),
 * p = p* rho c_s^2 (p* = sum_i g_i).  Any output may be NULL.  u is three
 * planes.  Host outputs synchronise the stream. */
lbm_status lbm_get_fields(lbm_t *s, float *phi, float *u, float *p, int on_device);

/* LBM_DIAG_COUNT doubles into host memory (see the LBM_DIAG_* indices);
 * synchronises the stream. */
lbm_status lbm_reduce(lbm_t *s, double *out);

/* Full state at time level t, pre-collision, in the natural population layout
 * above: h = h^{t+1} (q_phase planes; the phase field runs one step ahead, see
 * Algorithm 2), g = g^t (q_hydro planes), phi = phi^t.  Any output may be NULL.
 * lbm_set_state takes the same three arrays (none may be NULL) and makes them
 * the current state; it also marks the handle initialised.  Checkpoint and
 * restart use the pair. */
lbm_status lbm_get_state(lbm_t *s, float *h, float *g, float *phi, int on_device);
lbm_status lbm_set_state(lbm_t *s, const float *h, const float *g, const float *phi, int on_device);

/* Waits for the stream; returns LBM_ERR_DIVERGED once any step has produced a
 * non-finite phi or p*. */
lbm_status lbm_synchronize(lbm_t *s);

/* Number of time steps advanced since lbm_init_phase (or lbm_set_state). */
int64_t lbm_steps_done(const lbm_t *s);

/* Text of the last failure on this handle; with s == NULL, of the last failed
 * call without a handle (lbm_workspace_size, lbm_create,
 * lbm_reduce_state_noalloc) on the calling thread. */
const char *lbm_last_error(const lbm_t *s);

/* Releases the handle and, if the library allocated it, the workspace. */
void lbm_destroy(lbm_t *s);

/* ---- Batched stepping: many independent simulations advanced together -----
 *
 * A batch advances several independent problems (their own sizes, walls and
 * Section 3 parameters; one hydrodynamic lattice for all) by the coupled step
 * of Algorithm 2, each exactly as lbm_step would advance it alone: one launch
 * per time step (per group of up to 64 members) runs one thread block per entry
 * of a table of the members' cell tiles (32 x TY x TZ cells with one cell per
 * thread, or 32 x 4 x 2 with two).  Aimed at parameter
 * sweeps of small boxes, which alone cannot fill the GPU.
 *
 * Members are ordinary lbm_t handles owned by the batch (lbm_batch_member):
 * initialise them with lbm_init_phase or lbm_set_state, read them with
 * lbm_get_fields, lbm_reduce, lbm_get_state; do not lbm_step or lbm_destroy
 * them.  All members must be at the same time level when the batch steps
 * (LBM_ERR_STATE otherwise).  FP32 population storage only. */
typedef struct lbm_batch_t lbm_batch_t; /* opaque batch handle */

/* Device workspace for the batch's members: the sum over members of
 * lbm_workspace_size, each rounded up to a multiple of 256 bytes.  Host-only. */
lbm_status lbm_batch_workspace_size(int count, const lbm_domain *doms, const lbm_params *prms, size_t *bytes);

/* Creates a batch of count (1..65536) members from count domains and
 * parameter sets (validated as by lbm_create; every q_hydro equal, every
 * precision LBM_PRECISION_FP32, every phase_collision LBM_PHASE_SRT, every
 * kernel_form LBM_FORM_FUSED, every q_phase 15 and every member small enough
 * that (q_hydro - 1) * nx * ny * nz < 2^32, else LBM_ERR_ARG) on the current
 * CUDA device.
 * cuda_stream: stream for all of the batch's work (members included), NULL for
 * the legacy default stream (then no CUDA graphs are used).  workspace: device
 * buffer of lbm_batch_workspace_size() bytes, 256-byte aligned, owned by the
 * caller until lbm_batch_destroy; or NULL to let each member allocate its own.
 * The batch itself allocates its member and tile tables (a few bytes per tile).
 * Errors of this call read as lbm_last_error(NULL). */
lbm_status lbm_batch_create(lbm_batch_t **out, int count, const lbm_domain *doms, const lbm_params *prms,
                            void *cuda_stream, void *workspace, size_t workspace_bytes);

/* Number of members (0 for NULL). */
int lbm_batch_size(const lbm_batch_t *b);

/* Member i (0-based) of the batch, or NULL if i is out of range.  The handle
 * stays owned by the batch. */
lbm_t *lbm_batch_member(lbm_batch_t *b, int i);

/* Advances every member by n >= 0 coupled time steps.  Asynchronous.  On a
 * non-default stream, runs of 16 steps are replayed from CUDA graphs captured
 * on first use (so the first call of a run may take longer). */
lbm_status lbm_batch_step(lbm_batch_t *b, int64_t n);

/* Autotuner (the tile shapes and the halo staging of the batched step): for
 * each of 2 phi halo stagings (0: per-thread loads; 1: one TMA tensor copy per
 * block, walled faces mirrored in shared memory, per-thread loads for tiles on
 * a periodic face), 4 tile shapes (0, 1, 2: tiles of 32 x TY x TZ cells with one
 * cell per thread, (TY, TZ) = (4, 2), (8, 1), (2, 4); 3: tiles of 32 x 4 x 2
 * cells with two cells per thread, the LBM_FORM_FUSED_PAIR step) and 2 table
 * orders (0: member after member; 1: members' tiles dealt out round robin),
 * runs 1 + trial_steps batched steps, times the trial steps with CUDA events,
 * and keeps the fastest.  Candidate index: (halo * 4 + shape) * 2 + order.  The
 * trial steps are real time steps: every member advances by 1 + trial_steps per
 * timed candidate.  The TMA staging needs every member's nx to be a multiple of
 * 4 (and the CUDA driver's tensor-map support), shape 3 every member's nx even
 * and per-thread loads; candidates that do not apply are skipped and reported
 * as -1.  choice (may be NULL) receives the winner's index; ms_per_step (may be
 * NULL) receives the 16 times by index.  Synchronises the stream. */
lbm_status lbm_batch_tune(lbm_batch_t *b, int trial_steps, int *choice, double *ms_per_step);

/* Selects candidate `choice` of lbm_batch_tune (same index) without timing.
 * LBM_ERR_ARG if choice is outside 0..15; LBM_ERR_STATE, with the configuration
 * in use unchanged, if it asks for the TMA staging or the two-cell tiles and
 * these members do not allow them.  Host-only apart from uploading the tile
 * table (synchronises the stream). */
lbm_status lbm_batch_set_config(lbm_batch_t *b, int choice);

/* lbm_synchronize on every member: LBM_ERR_DIVERGED if any member produced a
 * non-finite phi or p*, LBM_ERR_CUDA if a TMA copy of a member's phi tile did
 * not complete (lbm_last_error on that member says which).  A block whose copy
 * did not complete within the bounded wait returns while the copy may still
 * land in shared memory that a later block of the same launch uses, so after
 * that error the state of every member of the batch and the results of that
 * launch are undefined: destroy the batch and create it again. */
lbm_status lbm_batch_synchronize(lbm_batch_t *b);

/* Text of the last failure of a batch call on b. */
const char *lbm_batch_last_error(const lbm_batch_t *b);

/* Releases the batch, its members and whatever they allocated. */
void lbm_batch_destroy(lbm_batch_t *b);

/* The LBM_DIAG_* diagnostics of a state that the caller holds in device memory,
 * computed without allocating any device memory.  The paper has no counterpart:
 * this serves callers that cannot allocate at this point -- a host application
 * whose memory pool already owns the GPU's free memory, or a time loop that must
 * not take the synchronisation cudaMalloc/cudaFree can cause.
 *   g, phi : device pointers to g^t (q_hydro planes, natural layout) and phi^t
 *            (nx*ny*nz floats), e.g. as lbm_get_state(..., on_device = 1) returns;
 *   out    : LBM_DIAG_COUNT doubles in host memory;
 *   cuda_stream : stream to run on (NULL: legacy default); synchronised on return.
 * Scratch space is a fixed array inside the library (about 786 KB per GPU, held
 * until the process exits): boxes of more than 134,217,728 cells (512^3) are
 * rejected with LBM_ERR_ARG.  The first call on a device looks up that array's
 * device address, so make that first call before any stream capture.  The lookup
 * is kept per device for the life of the process: it belongs to the device's
 * primary context, so after cudaDeviceReset the kept address is stale and this
 * entry point must not be called again in that process.  All calls
 * share the array and it keeps the last call's contents (each call overwrites
 * what it reads); calls that overlap on the GPU race on it, so the caller must
 * serialise them. */
lbm_status lbm_reduce_state_noalloc(const lbm_domain *dom, const lbm_params *prm, const float *g, const float *phi,
                                    double *out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
