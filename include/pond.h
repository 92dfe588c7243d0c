/*
 * libpond — GB300 (sm_103a) CUDA implementation of the particles-on-demand (PonD)
 * double-distribution-function BGK step for 2-D compressible flow, after
 * Hosseini, Bhadauria & Karlin, arXiv 2405.11489, Sec. III.A (and Sec. II for the
 * kinetic model).
 *
 * One time step per node (Sec. III.A): recover rho, rho u and the energy from the
 * populations (Sec. II); take the local frame lambda = (u, T) and the lattice
 * C_i = sqrt(T) c_i + u shifted and scaled from the Gauss-Hermite quadrature of Table I;
 * stream f and g semi-Lagrangianly from the departure points x - C_i dt, interpolating
 * the neighbours' populations after moving them into the receiving node's frame with the
 * reduced Grad transform (Eqs. gradGeneralTransform, propagationInterpolated); iterate
 * this predictor-corrector until the frame converges; relax f and g to their equilibria
 * (BGK, tau = mu / p, Eq. kin_visc).  The energy split is the total-energy split (Eq. Es,
 * first line) by default, the internal-energy split (second line, with the source term of
 * Eq. int_g_evolution) as an option.  The internal split's source is integrated along the
 * characteristics by the trapezoidal rule: the stored g is the post-collision g carried as
 * g - (Omega + G)/2, a node's internal energy is U = sum g + (1/2) sum G = sum g -
 * (1/2) rho T div u with div u at the new time level from a predictor pass (each node's f
 * streamed once in its previous frame; the step takes its first predictor-corrector iteration
 * from that pass), and the collision adds (1 - omega/2) G; a step of that split is three
 * launches (predictor, step, source).  Its reported temperature is the frame's.
 *
 * Units: lattice units (Sec. III), r = 1, dx = dt = 1, T_L = 1.
 *
 * Conventions for every entry point:
 *  - Return value: a pond_status_t (0 = POND_OK, negative = error).  Kernel-side outcomes
 *    (non-physical state, predictor-corrector non-convergence) are sticky: pond_step
 *    returns as soon as the work is enqueued, and the next synchronising call
 *    (pond_get_moments, pond_get_populations, pond_get_stats, pond_sync) reports them.
 *  - Fields are row-major [ny][nx] arrays of double (x fastest); population arrays are
 *    [Q][ny][nx] with population i = b * q1 + a (c_i = (c_a, c_b), q1 = 4 or 5).
 *  - Ownership: the caller owns every buffer it passes in (host or device), including the
 *    device workspace given to pond_create.  The library copies inputs, never keeps a
 *    pointer to a caller's input or output buffer beyond the call, and never frees caller
 *    memory.  pond_create allocates only the small host-side handle; the first
 *    synchronising call of a host thread allocates a 64-byte page-locked mirror of the
 *    status block for that thread's reads (kept for the thread's life).
 *  - Streams: all device work of a simulation is enqueued on the CUDA stream given to
 *    pond_create (NULL = the legacy default stream).
 *  - Thread safety: one pond_sim per host thread, or external synchronisation.
 *  - Device: the workspace's device must be current when calling into a pond_sim.
 */
#ifndef POND_H
#define POND_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    POND_OK = 0,
    POND_EINVAL = -1,          /* invalid argument or configuration */
    POND_ENOMEM = -2,          /* workspace too small */
    POND_ECUDA = -3,           /* a CUDA runtime call failed */
    POND_ENONPHYSICAL = -4,    /* rho <= 0, T <= 0 or NaN met at some node (state not repaired) */
    POND_ENOCONV = -5          /* predictor-corrector hit pc_max_iter at >= 1 node (state advanced) */
} pond_status_t;

enum { POND_D2Q16 = 16, POND_D2Q25 = 25 };                       /* Table I lattices */
enum { POND_SPLIT_TOTAL = 0, POND_SPLIT_INTERNAL = 1, POND_SPLIT_NT = 2 };   /* Eq. Es, lines 1-3 */
enum { POND_FP64 = 0, POND_MIXED_FP32 = 1, POND_MIXED_FP16 = 2, POND_MIXED_BF16 = 3 };
enum { POND_BC_PERIODIC = 0, POND_BC_OUTFLOW = 1, POND_BC_WALL = 2, POND_BC_INFLOW = 3 };

typedef struct {
    int32_t nx, ny;            /* grid; ny = 1 runs the quasi-1-D form (all y taps on row 0) */
    int32_t lattice;           /* POND_D2Q16 (default) or POND_D2Q25 */
    int32_t split;             /* POND_SPLIT_TOTAL (default), POND_SPLIT_INTERNAL or POND_SPLIT_NT
                                  (non-translational: E = sum g + sum v^2/2 f, g_eq = (U'/rho) f_eq;
                                  the paper's minimum lattice for it is D2Q25) */
    int32_t precision;         /* POND_FP64: FP64 storage and arithmetic.  POND_MIXED_*:
                                  FP32 arithmetic on deviations from a per-tile reference
                                  equilibrium, FP64 rho/u/T and frame update, non-equilibrium
                                  state stored in FP32 / FP16 / BF16 */
    int32_t interp_order;      /* 3: 4-point cubic Lagrange (default); 2: 3-point (Sec. III.A.2) */
    int32_t bc_x, bc_y;        /* POND_BC_PERIODIC (index mod n), POND_BC_OUTFLOW (clamp: zero-gradient
                                  copy of the edge node), POND_BC_WALL (not in the paper: every
                                  position beyond the wall holds the equilibrium at the wall's
                                  state, given in wall[]; the wall lies half a cell beyond the last
                                  node; not for y when ny = 1) or POND_BC_INFLOW (the prescribed
                                  conditions of the jet's inlet, Sec. III.C: the low side is
                                  prescribed like a wall, the high side is outflow; not for y when
                                  ny = 1).  A prescribed side's state may vary along it:
                                  pond_set_boundary_profile */
    double gamma;              /* adiabatic exponent, 1 < gamma <= 2 (c_v = 1/(gamma - 1)) */
    double mu;                 /* dynamic viscosity > 0; tau = mu / (rho T) per node */
    double pc_tol;             /* predictor-corrector tolerance on max(|du|/sqrt(T), |dT|/T) */
    int32_t pc_max_iter;       /* iteration cap (1..64) */
    int32_t pc_fixed_iters;    /* > 0: exactly this many iterations, no tolerance test */
    int32_t tile_x, tile_y;    /* 0 = automatic (32 x 8; 128 x 1 when ny = 1); otherwise the
                                  tile in nodes, tile_x * tile_y = 256 (128 x 1 when
                                  ny = 1) */
    int32_t halo;              /* 0 = automatic (5); the staged box is the tile plus
                                  2 * halo + 2 nodes per axis; stencils outside it are read
                                  from global memory (slower, same result) */
    int32_t grad_order;        /* Grad expansion order N of the frame transformation
                                  (Eq. gradGeneralTransform): 0 = the lattice's, which is the
                                  only value accepted: 3 on D2Q16, 4 on D2Q25 */
    double wall[4][4];         /* uniform states of the sides x-low, x-high, y-low, y-high:
                                  (u_x, u_y, T, rho), used on the prescribed sides (both sides
                                  of a POND_BC_WALL axis, the low side of a POND_BC_INFLOW axis;
                                  T > 0, rho > 0) */
} pond_config;

typedef struct {
    int64_t steps;             /* time steps taken since the last pond_set_state */
    int64_t node_updates;      /* nx * ny * steps */
    int64_t pc_iters_total;    /* sum over node updates of predictor-corrector iterations */
    int32_t pc_iters_max;      /* largest iteration count of any node update */
    int32_t status;            /* sticky kernel-side status (pond_status_t) */
    int64_t nonconv_updates;   /* node updates that hit pc_max_iter */
    int64_t first_bad_node;    /* first node (y * nx + x) found non-physical, or -1 */
    int64_t halo_fallbacks;    /* populations whose stencil left the staged tile (global gathers) */
} pond_stats;

typedef struct pond_sim pond_sim;

/* Fill *cfg with the defaults (D2Q16, total split, mixed FP32, cubic, periodic,
 * gamma 1.4, mu 1e-3, pc_tol 1e-6 (mixed) / 1e-12 (FP64), pc_max_iter 20) for nx x ny. */
int pond_config_default(pond_config *cfg, int32_t nx, int32_t ny);

/* Bytes of device workspace a simulation with this configuration needs (two copies of the
 * state, see pond_state_bytes, a status block, the prescribed sides' profiles and, for the
 * internal-energy split, its predictor pass's velocities and streamed coefficients: 96 bytes
 * per node in the mixed modes and 176 in FP64 on D2Q16, 136 and 256 on D2Q25).  For admission
 * by free HBM. */
int pond_workspace_bytes(const pond_config *cfg, size_t *bytes);

/* Create a simulation on the current device.  dev_workspace: caller-owned device memory
 * of at least pond_workspace_bytes bytes, 256-byte aligned; cuda_stream: a cudaStream_t
 * (or NULL).  *out receives the handle.  POND_EINVAL on a bad configuration,
 * POND_ENOMEM if bytes is too small. */
int pond_create(const pond_config *cfg, void *dev_workspace, size_t bytes, void *cuda_stream,
                pond_sim **out);

/* Set the macroscopic state: equilibrium populations f_i = rho w_i, g_i = g_eq_i in each
 * node's own frame (Sec. III.A).  rho, ux, uy, T: [ny][nx] doubles, host pointers
 * (on_device = 0) or device pointers (on_device = 1).  Requires rho > 0, T > 0 and finite
 * values: host input is checked after its copy to the device and before it replaces the
 * state (POND_EINVAL, state unchanged; the call synchronises the stream for this); device
 * input is checked by the next step.  Resets statistics and the sticky status. */
int pond_set_state(pond_sim *sim, const double *rho, const double *ux, const double *uy,
                   const double *T, int on_device);

/* Set populations directly: f, g [Q][ny][nx] in the frames (ux, uy, T) [ny][nx].  The
 * library keeps their Hermite coefficients up to total order 3 in each node's frame, which
 * is all that the frame transformation (N = 3) passes on.  Device pointers only
 * (on_device must be 1, else POND_EINVAL).  Resets statistics and the sticky status. */
int pond_set_populations(pond_sim *sim, const double *f, const double *g, const double *ux,
                         const double *uy, const double *T, int on_device);

/* Per-position states of a prescribed side (not in the paper; the jet's inlet of Sec. III.C
 * is prescribed over part of a side).  side: 0 x-low, 1 x-high, 2 y-low, 3 y-high; it must
 * be prescribed by the configuration (both sides of a POND_BC_WALL axis, the low side of a
 * POND_BC_INFLOW axis), else POND_EINVAL.  state: [n][4] (u_x, u_y, T, rho) along the side,
 * n = ny for the x sides and nx for the y sides; the ghost position beyond the side at
 * coordinate k along it (clamped to 0 .. n - 1; corners belong to the y sides) holds the
 * equilibrium at state[k].  NULL restores the uniform state cfg->wall[side] (the state at
 * pond_create).  Host (on_device = 0; checked: T > 0, rho > 0, finite, else POND_EINVAL)
 * or device pointers (unchecked: a non-physical state shows in the next step's status).
 * The library copies the states into the workspace; every later step, batched step and
 * captured graph replay reads them.  Not part of pond_export_state. */
int pond_set_boundary_profile(pond_sim *sim, int32_t side, const double *state, int on_device);

/* Advance nsteps >= 0 time steps, asynchronously on the simulation's stream. */
int pond_step(pond_sim *sim, int32_t nsteps);

/* Moments of the current populations: rho, ux, uy, T [ny][nx] (any pointer may be NULL).
 * Host (on_device = 0) or device pointers; page-locked host buffers (cudaHostAlloc,
 * cudaHostRegister) are written by the kernel in place, other host memory through a staging
 * copy.  Synchronises the stream and returns the sticky status.  In FP64 the moments are
 * summed in FP64 (Sec. II); in the mixed modes the contributions of the stored FP32 (or
 * FP16/BF16) non-equilibrium coefficients are formed in FP32 and added to the FP64 frame. */
int pond_get_moments(pond_sim *sim, double *rho, double *ux, double *uy, double *T,
                     int on_device);

/* Current populations f, g [Q][ny][nx] and their frames (ux, uy, T) [ny][nx], each node in
 * its own frame (f_i = w_i sum A_pq He_p(c_ia) He_q(c_ib) / (p! q!)).  Device pointers only
 * (on_device must be 1).  Synchronises; returns the sticky status. */
int pond_get_populations(pond_sim *sim, double *f, double *g, double *ux, double *uy,
                         double *T, int on_device);

/* Raw state (checkpoint / resume).  The state is mac = [4][ny][nx] FP64 (rho, u_x, u_y, T) and
 * neq = [P][ny][nx] in the storage type of cfg->precision (8, 4, 2 or 2 bytes): the
 * non-equilibrium Hermite coefficients of total order <= N (N = 3 on D2Q16, 4 on D2Q25) of f
 * (all but A_00) and of g (B_pq - B_pq^eq), in each node's own frame,
 * A_pq = sum_i f_i He_p(c_ia) He_q(c_ib) (Sec. III.A.1), slots ordered by total order and then
 * by q: (p,q) = 00 | 10 01 | 20 11 02 | 30 21 12 03 | 40 31 22 13 04; P = 19 for N = 3
 * (9 + 10), 29 for N = 4 (14 + 15).
 * pond_state_bytes gives the two array sizes.  Export copies the current state into the
 * caller's buffers (host or device) and synchronises; import copies it in (statistics and
 * sticky status reset).  A checkpoint resumes bit-identically on the same build. */
int pond_state_bytes(const pond_config *cfg, size_t *mac_bytes, size_t *neq_bytes);
int pond_export_state(pond_sim *sim, double *mac, void *neq, int on_device);
int pond_import_state(pond_sim *sim, const double *mac, const void *neq, int on_device);

/* Statistics since the last pond_set_state*.  Synchronises; returns the sticky status. */
int pond_get_stats(pond_sim *sim, pond_stats *stats);

/* Wait for the simulation's queued work; returns the sticky status. */
int pond_sync(pond_sim *sim);

/* Free the handle (not the caller's workspace).  Waits for queued work first. */
int pond_destroy(pond_sim *sim);

/* Batched stepping (many simulations, one kernel launch per time step).
 *
 * A batch advances count simulations together: every time step is one launch of the step
 * kernel over the tiles of all of them (plus one launch each of the internal split's predictor
 * and source passes if any member uses that split), so uneven cases share the GPU without per-case launches or
 * tail effects.  The members must share precision, lattice, interpolation order, the 1-D
 * (ny = 1) or 2-D class and the tile configuration; grid size, boundaries, split, gamma, mu
 * and the predictor-corrector settings may differ.  dev_workspace (caller-owned device
 * memory of pond_batch_workspace_bytes(count), 256-byte aligned) holds the case table.  The
 * members' own handles stay valid and see the batch's steps (pond_get_moments etc.), but a
 * member must not be stepped through pond_step while its batch exists.  The batch works on
 * cuda_stream and orders itself with events: each pond_batch_step waits for the work already
 * queued on the members' streams, and later work on those streams waits for the batch.
 * pond_batch_use_graph(batch, k), k even and > 0, captures k time steps into a CUDA graph
 * that pond_batch_step then replays (k = 0 returns to plain launches); it needs a non-NULL
 * stream.  Errors: POND_EINVAL for mismatched members or bad arguments, POND_ENOMEM for a
 * small workspace. */
typedef struct pond_batch pond_batch;
int pond_batch_workspace_bytes(int32_t count, size_t *bytes);
int pond_batch_create(pond_sim *const *sims, int32_t count, void *dev_workspace, size_t bytes,
                      void *cuda_stream, pond_batch **out);
int pond_batch_step(pond_batch *batch, int32_t nsteps);
/* pond_set_state for every member at once: rho[i], ux[i], uy[i], T[i] are member i's
 * [ny][nx] fields (count pointers each, host or device as on_device says).  The same checks
 * and effects as pond_set_state on each member, on the batch's stream and ordered with the
 * members' streams like pond_batch_step; host input is checked on the device with one
 * synchronisation for the whole batch, and if any member's input is rejected no member's
 * state changes (POND_EINVAL).  When every member's four host arrays are page-locked they are
 * read in place by one kernel per 64 members, which checks and stages them; other host
 * memory is copied first.  The status blocks are cleared, and the equilibria set, by one
 * launch each per 64 members. */
int pond_batch_set_state(pond_batch *batch, const double *const *rho, const double *const *ux,
                         const double *const *uy, const double *const *T, int on_device);
/* pond_get_moments for every member at once (any of the four pointer arrays may be NULL, and
 * any member's pointer in them): one synchronisation of the batch's stream for all members;
 * returns the worst member status (POND_ENONPHYSICAL before POND_ENOCONV), each member's own
 * status stays available through pond_get_stats.  Device buffers, and page-locked host
 * buffers when every given buffer is page-locked, are written in place by one kernel per 64
 * members; otherwise each member's moments pass through a staging copy.  The first batched
 * read-back of a host thread allocates a
 * page-locked array of status blocks for it (grown to the largest batch and kept for the
 * thread's life). */
int pond_batch_get_moments(pond_batch *batch, double *const *rho, double *const *ux,
                           double *const *uy, double *const *T, int on_device);
int pond_batch_use_graph(pond_batch *batch, int32_t steps_per_graph);
int pond_batch_destroy(pond_batch *batch);

/* Launch shapes and autotuning.  (No counterpart in the paper: the paper gives no
 * implementation; this tunes the staging of its interpolation stencils, Sec. III.A.2.)
 *
 * The step kernel runs one CTA per tile of 256 nodes (128 on quasi-1-D grids, two CTAs per
 * SM) and stages, per tile, the source nodes
 * of its interpolation stencils in shared memory; the staged box holds the tile plus
 * 2 * halo + 2 nodes per axis, and stencils that leave it are gathered from global memory.
 * The shape (tile_x, tile_y, halo) changes speed only, never results beyond rounding (the
 * tile's centre node is the reference of the FP32 deviation arithmetic).
 *  - pond_get_launch: the current shape of sim (candidates = 0, ms_per_step = 0).
 *  - pond_set_launch: set sim's shape (0 = default, as in pond_config); POND_EINVAL if
 *    tile_x * tile_y != 256 (on quasi-1-D grids: the tile is not 128 x 1), tile_x is odd,
 *    or the box does not fit shared memory.
 *  - pond_autotune: time every candidate shape -- tiles 32x8, 16x16, 64x4, 128x2, 8x32 on
 *    2-D grids (128x1 on quasi-1-D ones) times halos 4, 5, 6, 8 -- by running
 *    1 + steps time steps of a copy of sim's current state in dev_scratch (caller-owned
 *    device memory of pond_workspace_bytes(cfg) bytes, 256-byte aligned) on sim's stream,
 *    time the three fastest twice more (each keeps its best time), and return the fastest
 *    in *out (candidates = shapes timed, ms_per_step its best time per step).  sim's own state and statistics are untouched; kernel-side statuses of the
 *    copy (POND_ENOCONV, POND_ENONPHYSICAL) do not rule a shape out.  Results are cached per class
 *    (precision, lattice, interpolation order, split, 1-D or 2-D, boundaries, and nx, ny
 *    rounded up to powers of two) for the life of the process: a later call for the same
 *    class returns the cached shape with candidates = 0 and touches neither the GPU nor
 *    dev_scratch (which may then be NULL).  flags: POND_TUNE_APPLY also sets the shape on
 *    sim; POND_TUNE_RETIME times again even if the class is cached.  Synchronises sim's
 *    stream.  Errors: POND_EINVAL (bad arguments, or no candidate could run),
 *    POND_ENOMEM (small scratch), POND_ECUDA.
 *  - pond_autotune_clear: empty the cache. */
typedef struct {
    int32_t tile_x, tile_y;    /* tile in nodes */
    int32_t halo;              /* staged box = tile + 2 * halo + 2 per axis */
    int32_t candidates;        /* shapes timed by this call (0: current or cached shape) */
    double ms_per_step;        /* time per step of the chosen shape when it was timed */
} pond_tuning;
enum { POND_TUNE_APPLY = 1, POND_TUNE_RETIME = 2 };
int pond_get_launch(pond_sim *sim, pond_tuning *out);
int pond_set_launch(pond_sim *sim, int32_t tile_x, int32_t tile_y, int32_t halo);
int pond_autotune(pond_sim *sim, void *dev_scratch, size_t bytes, int32_t steps, int32_t flags,
                  pond_tuning *out);
void pond_autotune_clear(void);

/* Allocation-free stepping.  (No counterpart in the paper: this is plumbing for callers.)
 *
 * Some callers cannot allocate device memory: an application that owns all GPU memory
 * through its own pool and forbids any other allocation; a real-time loop that cannot
 * afford the latency and implicit device synchronisation of cudaMalloc; a plugin or
 * foreign-language host that holds only the state buffers it was given.  Such a caller
 * cannot provide the workspace that pond_create needs.  pond_step_static advances nsteps
 * time steps of a raw state (the layout of pond_state_bytes / pond_export_state) that lives
 * in the caller's own device buffers mac and neq, in place, on cuda_stream, with the same
 * kernels as pond_step, and allocates nothing: the second copy of the state and the status
 * block live in one file-scope device array of the library, POND_STATIC_SCRATCH_BYTES
 * (16 MiB) on every GPU that loads the library, held until the process exits.
 *  - Size limit: the state must fit that array, state bytes = align256(4*8*N) +
 *    align256(P*s*N) + 256 with N = nx*ny, P = 19 (D2Q16) or 29 (D2Q25) and s = 8/4/2/2
 *    bytes (FP64/FP32/FP16/BF16), i.e. N <= 91 178 / 63 548 (FP64), 155 341 / 113 357
 *    (FP32), 239 669 / 186 408 (FP16/BF16) on D2Q16 / D2Q25; the internal-energy split adds
 *    align256 of its predictor region (96 / 176 bytes per node on D2Q16 in the mixed / FP64
 *    modes, 136 / 256 on D2Q25).  Larger grids return POND_ENOMEM without touching the GPU.
 *  - Set-up: the first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) and the SM count, and the first call for each kernel variant
 *    (precision, lattice, 1-D or 2-D, interpolation order, launch shape) sets the step
 *    kernel's shared-memory limit; make those first calls before any stream capture on that
 *    device.  Later calls query only the current device and context (cudaGetDevice and the
 *    driver's context ID) and enqueue the status clear and the kernels.  If the current
 *    context changes (after cudaDeviceReset, or another context made current), the next
 *    call repeats the set-up.
 *  - Every call uses the same array and it keeps the last call's contents; the status
 *    block is cleared at the start of each call.  Calls that overlap on the GPU (other
 *    streams, other host threads) race on the array: serialise them.
 *  - stats: if non-NULL the call synchronises cuda_stream, fills *stats for this call and
 *    returns the sticky status; if NULL it returns once the work is enqueued, and the
 *    kernel-side outcomes of this call (POND_ENONPHYSICAL, POND_ENOCONV) are not reported
 *    at all: the next call clears the status block. */
#define POND_STATIC_SCRATCH_BYTES (16u << 20)
int pond_step_static(const pond_config *cfg, double *mac, void *neq, int32_t nsteps,
                     void *cuda_stream, pond_stats *stats);

/* ALU peak measurement.  (No counterpart in the paper: the measured denominator of the step
 * kernel's roofline, which is bound by the CUDA-core FP32 pipe, or the FP64 pipe in the
 * FP64 mode.)  Runs one launch of independent FMA chains, 4 blocks of 256 threads per SM,
 * each thread 8 chains of 16 * iters dependent FMAs, on cuda_stream (NULL = legacy default
 * stream) on the current device, and waits for it.  fp64: 0 = FP32 FMAs, 1 = FP64 FMAs.
 * On success *flop = the flops executed (2 per FMA) and *ms = their CUDA-event time; divide
 * for the rate.  Allocates nothing.  Errors: POND_EINVAL (iters <= 0, fp64 not 0 or 1, a
 * NULL output), POND_ECUDA. */
int pond_alu_peak(int32_t fp64, int32_t iters, void *cuda_stream, double *flop, float *ms);

/* Static description of a status code. */
const char *pond_strerror(int status);

/* Library version string. */
const char *pond_version(void);

#ifdef __cplusplus
}
#endif
#endif /* POND_H */
