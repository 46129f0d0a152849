/*
 * wblbe.h - C ABI of the GB300 (sm_103a) library for the well-balanced
 * lattice Boltzmann equation of Guo, "Well-balanced lattice Boltzmann
 * equation for two-phase flows" (arXiv 2012.11075), with the standard LBE of
 * its Sec. II as the comparison scheme.
 *
 * The method (lattice units dx = dt = c = 1, cs^2 = 1/3, periodic D2Q9):
 *   f_i(x + c_i, t + 1) = f_i - (f_i - f_i^eq)/tau + (1 - 1/(2 tau)) F_i
 *                                                             (Eq. D2Q9)
 *   rho = sum_i f_i,  rho u = sum_i c_i f_i + F/2             (Eq. rhoU)
 *   mu  = mu_0(rho) - kappa lap(rho),
 *   mu_0 = d/drho [beta (rho - rho_l)^2 (rho - rho_g)^2]      (Eq. doubleWell)
 *   well-balanced: f^eq of Eq. mFeq, F = -rho grad(mu) (Eq. mF), F_i of Eq. mFi
 *   standard:      f^eq of Eq. feq,  F = grad(cs^2 rho) - rho grad(mu)
 *                  (potential form, Sec. II), F_i of Eq. Fi.
 * Gradients and the Laplacian are the isotropic central stencils
 *   grad(phi) = 3 sum_i w_i c_i phi(x + c_i),
 *   lap(phi)  = 6 sum_i w_i (phi(x + c_i) - phi(x)),
 * which reduce to the 1D central forms of Sec. II.
 *
 * Conventions for every function below:
 *  - Every call returns a wblbe_status; nothing throws across the ABI.  On a
 *    non-OK status, wblbe_last_error(h) gives a one-line reason.
 *  - Handles are not thread-safe: one host thread drives a handle at a time.
 *  - Scalar fields are row-major [ny][nx] float64 (x fastest); population
 *    arrays are [9][ny][nx] float64, direction order
 *    c0=(0,0) c1=(1,0) c2=(0,1) c3=(-1,0) c4=(0,-1) c5=(1,1) c6=(-1,1)
 *    c7=(-1,-1) c8=(1,-1).  Populations are f_i(x, t): after streaming,
 *    before collision (the left-hand side of Eq. D2Q9 at time t).
 *  - Pointers flagged "on_device" are device addresses on the current CUDA
 *    device; otherwise they are host addresses.  All arrays are owned by the
 *    caller.  The library allocates no device memory: the caller passes one
 *    device workspace (for example a torch uint8 tensor) at creation and
 *    keeps it alive until wblbe_destroy.
 *  - Work is issued on the stream given at creation.  wblbe_step is
 *    asynchronous; functions that return data to host memory synchronise the
 *    stream before returning.
 */
#ifndef WBLBE_H
#define WBLBE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wblbe_ctx* wblbe_handle;

typedef enum {
  WBLBE_OK = 0,
  WBLBE_EINVAL = 1,        /* bad argument or parameter set                 */
  WBLBE_ENOMEM = 2,        /* workspace too small / no free slot or budget  */
  WBLBE_ECUDA = 3,         /* a CUDA runtime call failed                    */
  WBLBE_EUNSTABLE = 4,     /* a non-finite rho, u or mu was seen            */
  WBLBE_ETIMEOUT = 5,      /* a bounded device wait gave up                 */
  WBLBE_ENOTCONVERGED = 6  /* max_steps reached; the state is still valid   */
} wblbe_status;

/* Scheme: the standard LBE of Sec. II (potential-form force, forcing term
 * Eq. Fi) or the well-balanced LBE of Sec. III; and two variants of the
 * standard LBE that Sec. II compares with, for single lattices only (the
 * batch API rejects them with WBLBE_EINVAL):
 *   WBLBE_STANDARD_PRESSURE: pressure-form force
 *     F = grad(cs^2 rho - p_0) + kappa rho grad(lap rho) (Sec. II; the paper
 *     prints "- kappa grad(lap rho)", which would not equal the potential
 *     form it is said to equal);
 *   WBLBE_STANDARD_TEXTBOOK: potential-form force with the forcing term of
 *     Guo's textbook quoted in Sec. II, F_i = (c_i - u).F f_i^eq/(cs^2 rho);
 *   WBLBE_STANDARD_E6 (FP64 only): potential-form force whose gradients use
 *     the radius-2 stencil with moments isotropic to sixth order (weights
 *     4/15, 1/10, 1/120 on |e|^2 = 1, 2, 4) - Sec. II's "higher-order
 *     discretisation of F", for which the paper names no stencil.
 * All use the standard equilibrium Eq. feq (and its FP32 shift). */
enum { WBLBE_STANDARD = 0, WBLBE_WELL_BALANCED = 1, WBLBE_STANDARD_PRESSURE = 2,
       WBLBE_STANDARD_TEXTBOOK = 3, WBLBE_STANDARD_E6 = 4 };

/* Storage/arithmetic precision.
 * WBLBE_FP64: populations stored and updated in float64 (for the
 *   well-balanced scheme as deviations from the constant rho0 vector
 *   s_0 = -(1-w_0) rho0, s_i = w_i rho0, the shift below at rho_ref = 0; the
 *   update carries it unchanged, and get/set_populations use f_i itself).
 * WBLBE_FP32_SHIFTED: populations stored as float32 deviations
 *   g_i = f_i - s_i from the scheme's rest equilibrium s_i at rho_ref
 *   (standard: s_i = w_i rho_ref; well-balanced: s_0 = rho_ref - (1-w_0) rho0,
 *   s_i = w_i rho0), arithmetic in float32, reductions in float64.  The shift
 *   is exact in real arithmetic: sum_i s_i = rho_ref and a uniform s_i is
 *   invariant under streaming.  In the well-balanced scheme the rest
 *   population is taken from the node's exact mass balance and rounded
 *   stochastically (zero-mean rounding whose random bits come from a
 *   counter-based hash of the node and the time step, so results do not
 *   depend on the launch shape, batching or a slab split; see
 *   wblbe_set_step_count).  After 1e5 steps of a 256^2 droplet the mass is
 *   within about 1e-8 of its start, the droplet within 1e-4 lattice units of
 *   the FP64 run's position, the bulk densities within 1e-6 and the Laplace
 *   jump within 1e-4 of FP64, and max|u| near 1e-8.  Equilibria at
 *   round-off velocity need WBLBE_FP64. */
enum { WBLBE_FP64 = 0, WBLBE_FP32_SHIFTED = 1 };

/* The paper's statement of the problem (Sec. IV): lattice nx x ny (periodic),
 * relaxation time tau (> 1/2), interface parameter kappa (>= 0), double-well
 * height beta (> 0) and saturation densities rho_l > rho_g > 0
 * (Eq. doubleWell); rho0 is the numerical constant of Eq. mFeq (the paper
 * uses 0; only the well-balanced scheme reads it); rho_ref is the FP32 shift
 * density (NaN selects rho_g, which gives the low-density phase the finest
 * resolution of the stored deviations; ignored in FP64). */
typedef struct {
  int32_t nx, ny;
  double tau, kappa, beta, rho_l, rho_g;
  double rho0;
  double rho_ref;
  int32_t scheme;     /* WBLBE_STANDARD .. WBLBE_STANDARD_E6    */
  int32_t precision;  /* WBLBE_FP64 | WBLBE_FP32_SHIFTED        */
} wblbe_params;

/* Diagnostics of Sec. IV computed from the state f(t) at step `step`:
 * mass = sum rho, its drift relative to the mass after wblbe_init_rho /
 * wblbe_set_populations, max |u| (u of Eq. rhoU), min and max of mu,
 * kinetic energy E = 1/2 sum rho |u|^2, and a flag set if any rho, u or mu
 * was not finite.  All accumulated in float64. */
typedef struct {
  int64_t step;
  double mass, mass_drift_rel, umax, mu_min, mu_max, kinetic;
  int32_t nonfinite;
} wblbe_stats;

/* Launch shape of the fused step kernel: tile_x lattice columns per CTA
 * (32, 64, 128 or 256) and rows_per_cta rows marched by each CTA (>= 1).
 * Results do not depend on it. */
typedef struct {
  int32_t tile_x;
  int32_t rows_per_cta;
} wblbe_launch;

/* Device workspace bytes a handle with these parameters needs; 0 if the
 * parameters are invalid.  Layout: two population buffers, one float64 field
 * of staging, reduction partials and a stats record, each 256-byte aligned. */
size_t wblbe_workspace_bytes(const wblbe_params* params);

/* Create a handle.  dev_workspace: device pointer, 256-byte aligned, at
 * least wblbe_workspace_bytes(params) bytes, borrowed until wblbe_destroy.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).  The state is
 * undefined until wblbe_init_rho or wblbe_set_populations.
 * EINVAL: bad params, NULL out, misaligned or short workspace. */
wblbe_status wblbe_create(const wblbe_params* params, void* dev_workspace,
                          size_t workspace_bytes, void* cuda_stream,
                          wblbe_handle* out);

/* Change tau, kappa, beta, rho_l, rho_g, rho0 or the scheme between steps.
 * Changing nx, ny or precision, or anything that moves the storage shift
 * (rho_ref and the scheme in FP32; rho0 of the well-balanced scheme in both
 * precisions), returns EINVAL: the stored state depends on them. */
wblbe_status wblbe_set_params(wblbe_handle h, const wblbe_params* params);

/* Choose the launch shape (see wblbe_launch).  EINVAL on unsupported
 * values.  The default is picked from the lattice size at creation. */
wblbe_status wblbe_set_launch(wblbe_handle h, const wblbe_launch* launch);
wblbe_status wblbe_get_launch(wblbe_handle h, wblbe_launch* launch);

/* Initial state (Sec. IV): u = 0 and f_i = f_i^eq(rho, u = 0) of the
 * handle's scheme.  rho: [ny][nx] float64, host or device (rho_on_device).
 * Resets the step counter and the reference mass. */
wblbe_status wblbe_init_rho(wblbe_handle h, const double* rho,
                            int32_t rho_on_device);

/* Advance nsteps >= 0 time steps of Eq. D2Q9 (collision, streaming,
 * periodic boundaries).  Asynchronous on the handle's stream; repeated
 * chunks are replayed from a captured CUDA graph.  On ECUDA the step count
 * (wblbe_step_count) includes the steps issued before the failing launch. */
wblbe_status wblbe_step(wblbe_handle h, int64_t nsteps);

/* Step until max|u| < umax_tol, testing every check_every steps (> 0), or
 * until max_steps further steps were taken.  Blocking.  *steps_done (may be
 * NULL) receives the steps taken by this call and *out (may be NULL) the
 * stats of the last check.  Returns OK on convergence, ENOTCONVERGED at
 * max_steps, EUNSTABLE on a non-finite value. */
wblbe_status wblbe_run_until_equilibrium(wblbe_handle h, double umax_tol,
                                         int64_t max_steps,
                                         int64_t check_every,
                                         int64_t* steps_done,
                                         wblbe_stats* out);

/* Macroscopic fields of the current state f(t): rho, u (Eq. rhoU), mu,
 * as [ny][nx] float64 (each pointer may be NULL), on the host or device
 * (out_on_device), and the stats (may be NULL).  Synchronises the stream. */
wblbe_status wblbe_moments(wblbe_handle h, double* rho, double* ux,
                           double* uy, double* mu, int32_t out_on_device,
                           wblbe_stats* stats);

/* Copy the populations f_i(x, t) out as [9][ny][nx] float64 (unshifted), or
 * replace them (which resets the reference mass).  Synchronises. */
wblbe_status wblbe_get_populations(wblbe_handle h, double* f,
                                   int32_t on_device);
wblbe_status wblbe_set_populations(wblbe_handle h, const double* f,
                                   int32_t on_device);

/* Number of steps taken since the last init, and the number of kernels this
 * handle has launched (graph replays count every kernel in the graph). */
int64_t wblbe_step_count(wblbe_handle h);
int64_t wblbe_kernel_launches(wblbe_handle h);

/* Set the step counter (>= 0), e.g. after wblbe_set_populations when
 * resuming a checkpoint.  In WBLBE_FP32_SHIFTED storage with the
 * well-balanced scheme the counter also seeds the stochastic rounding of the
 * rest population (see WBLBE_FP32_SHIFTED), so a resumed run that restores
 * it repeats the rounding decisions of the run it continues.  EINVAL on a
 * NULL handle or a negative step. */
wblbe_status wblbe_set_step_count(wblbe_handle h, int64_t step);

/* Bytes of device scratch that wblbe_run_sequence needs for these params:
 * two input and two output float64 density fields plus four statistics
 * records.  0 for NULL or non-positive sizes. */
size_t wblbe_sequence_scratch_bytes(const wblbe_params* params);

/* Relax n independent initial states one after another with the host
 * copies overlapped: for each k, as wblbe_init_rho(rho_in[k], host), then
 * wblbe_step(nsteps), then wblbe_moments into rho_out[k] (host) and
 * stats[k] (may be NULL): the same results, bit for bit, as those calls
 * made one state at a time (Eq. D2Q9 from f = f^eq(rho, 0), Eq. rhoU).
 * State k + 1's density is copied in on a second stream while state k is
 * computed, and state k's density and statistics are copied out on a third
 * while state k + 1 is computed; the copies overlap the computation only
 * when rho_in and rho_out point to page-locked memory.
 * rho_in, rho_out: n host pointers to [ny][nx] float64 fields (the same
 * pointer may repeat; rho_out[k] is written when the call returns).
 * scratch: caller-owned device memory of wblbe_sequence_scratch_bytes()
 * bytes, 256-byte aligned, not in use by other work.  The call creates two
 * streams, eight events and a page-locked host buffer of 96 bytes per state
 * (the statistics records) and releases them before it returns.
 * Synchronises; the handle then holds the last state (its mass reference
 * that state's initial mass).  EINVAL: NULL handle or pointer, n < 0,
 * nsteps < 0, short or misaligned scratch; ECUDA: a failed launch, copy or
 * stream/event creation (work already issued is drained first; rho_out and
 * stats are then incomplete). */
wblbe_status wblbe_run_sequence(wblbe_handle h, int32_t n, const double* const* rho_in,
                                int64_t nsteps, double* const* rho_out, wblbe_stats* stats,
                                void* scratch, size_t scratch_bytes);

/* Release the handle (the workspace stays the caller's).  NULL -> EINVAL.
 * Synchronises the stream first. */
wblbe_status wblbe_destroy(wblbe_handle h);

/* Last error message of h, or of the calling thread when h is NULL. */
const char* wblbe_last_error(wblbe_handle h);

/* ---- batched cases and serving -------------------------------------------
 * A batch keeps many independent cases (each its own lattice size and
 * parameters, one scheme and precision for the whole batch) resident on the
 * device and advances all running cases together with one persistent kernel
 * per launch: the cases are cut into tiles of tile_x columns by about
 * rows_per_tile rows; a launch advances every running case by
 * steps_per_launch steps, tiles waiting (bounded) only for the neighbouring
 * tiles their halo reads.  Results are bit-identical to a wblbe_create
 * handle run alone.  Launches are replayed from a captured CUDA graph.
 * Memory: one caller workspace = control region + arena; each admitted case
 * takes wblbe_batch_case_bytes() of the arena until it is retired. */
typedef struct wblbe_batch* wblbe_batch_handle;

typedef struct {
  int32_t tile_x;            /* 32, 64, 128 or 256                         */
  int32_t rows_per_tile;     /* >= 4; rows are split into near-equal runs  */
  int32_t steps_per_launch;  /* >= 1 lattice steps per persistent launch   */
} wblbe_batch_config;

enum {
  WBLBE_CASE_RUNNING = 0,    /* being advanced                             */
  WBLBE_CASE_CONVERGED = 1,  /* max|u| fell below its tolerance            */
  WBLBE_CASE_MAXSTEPS = 2,   /* reached its step budget                    */
  WBLBE_CASE_UNSTABLE = 3    /* a non-finite value appeared                */
};

typedef struct {
  int64_t case_id;
  int32_t state;             /* WBLBE_CASE_*                               */
  int64_t steps;
  wblbe_stats stats;         /* at the last check (end of a launch group)  */
} wblbe_case_info;

/* Workspace bytes for a batch: control region for max_cases cases,
 * max_tiles tiles, cases of at most max_case_nodes nodes, plus arena_bytes of
 * arena.  0 on invalid arguments. */
size_t wblbe_batch_workspace_bytes(int32_t max_cases, int32_t max_tiles,
                                   int64_t max_case_nodes, size_t arena_bytes);

/* Arena bytes one case needs (two buffers with ghost columns); 0 if invalid. */
size_t wblbe_batch_case_bytes(const wblbe_params* params);

/* Create a batch on the current device.  dev_workspace: 256-byte aligned,
 * borrowed until destroy.  EINVAL / ENOMEM (workspace below the control
 * region) / ECUDA. */
wblbe_status wblbe_batch_create(int32_t scheme, int32_t precision,
                                int32_t max_cases, int32_t max_tiles,
                                int64_t max_case_nodes, void* dev_workspace,
                                size_t workspace_bytes, void* cuda_stream,
                                const wblbe_batch_config* config,
                                wblbe_batch_handle* out);
wblbe_status wblbe_batch_set_config(wblbe_batch_handle b,
                                    const wblbe_batch_config* config);
wblbe_status wblbe_batch_get_config(wblbe_batch_handle b,
                                    wblbe_batch_config* config);

/* Spins (about 64 ns each) a tile waits for a neighbour before the launch
 * gives up with WBLBE_ETIMEOUT (default 2^22).  Small values exist to
 * exercise that path. */
wblbe_status wblbe_batch_set_wait_limit(wblbe_batch_handle b, int64_t spins);

/* Admit a case: params (scheme/precision of the batch, nx, ny >= 8),
 * initial density rho ([ny][nx] float64, host), the max|u| tolerance that
 * counts as equilibrium and a step budget.  The case starts at rest,
 * f = f^eq(rho, 0).  ENOMEM when no case slot, arena range or tile-table room
 * is free: the caller keeps the request queued and retries after a retire.
 * On any error the case is not admitted: its slot and arena range stay free. */
wblbe_status wblbe_batch_admit(wblbe_batch_handle b, const wblbe_params* params,
                               const double* rho, double umax_tol,
                               int64_t max_steps, int64_t* case_id);

/* Run up to `launches` persistent launches, each advancing every running
 * case by steps_per_launch steps.  After every launch the statistics of the
 * running cases (of the state the launch's last step started from) are read
 * and the cases that converged, reached their step budget (checked at launch
 * boundaries, so a budget that is not a multiple of steps_per_launch is
 * overrun by less than one launch) or became unstable stop and leave the
 * next launch.  Blocking.  ETIMEOUT if a tile wait gave up (the batch state
 * is then invalid). */
wblbe_status wblbe_batch_advance(wblbe_batch_handle b, int32_t launches);

/* Ids of cases that stopped since the last poll (at most cap). */
wblbe_status wblbe_batch_poll(wblbe_batch_handle b, int64_t* ids, int32_t cap,
                              int32_t* n_done);
wblbe_status wblbe_batch_case_info(wblbe_batch_handle b, int64_t case_id,
                                   wblbe_case_info* info);

/* Macroscopic fields ([ny][nx] float64 host arrays, any may be NULL) and
 * stats of a resident case; populations f_i(x, t) as [9][ny][nx] float64. */
wblbe_status wblbe_batch_fetch(wblbe_batch_handle b, int64_t case_id,
                               double* rho, double* ux, double* uy, double* mu,
                               wblbe_stats* stats);
wblbe_status wblbe_batch_get_populations(wblbe_batch_handle b, int64_t case_id,
                                         double* f);

/* Free a case's slot, arena range and tiles. */
wblbe_status wblbe_batch_retire(wblbe_batch_handle b, int64_t case_id);

/* Cases resident and running, tiles of the running cases, free arena bytes
 * (any pointer may be NULL). */
wblbe_status wblbe_batch_counts(wblbe_batch_handle b, int32_t* resident,
                                int32_t* running, int32_t* tiles,
                                size_t* arena_free);
int64_t wblbe_batch_kernel_launches(wblbe_batch_handle b);
wblbe_status wblbe_batch_destroy(wblbe_batch_handle b);
const char* wblbe_batch_last_error(wblbe_batch_handle b);

/* ---- one lattice split into row slabs ------------------------------------
 * The update of Eq. D2Q9 is local: one step of a node reads the
 * post-collision populations of the previous step within 3 nodes of it (the
 * pulled populations, the densities that mu and its gradient need: Sec. II).
 * So a lattice can be split into slabs of whole rows, each advanced from its
 * own rows and 3 ghost rows on each side, with one exchange of ghost rows
 * per step.  These entry points do that on one device: nslabs slabs of
 * near-equal row counts (boundaries on even rows, every slab >= 3 rows),
 * stepped by the single-lattice kernels, the slabs' launches side by side
 * on streams the handle creates (forked from and joined back into the
 * caller's stream by events), and exchanged by one copy kernel per step,
 * with results equal bit for bit to a wblbe_create handle of the same
 * parameters (schemes 0-3; the E6 variant is refused).  Chunks of 16 steps
 * replay from a captured CUDA graph.  Conventions, arrays, workspace and
 * stream rules are those of the single-lattice API; the handle owns its
 * extra streams and events and releases them in wblbe_slabs_destroy. */
typedef struct wblbe_slabs* wblbe_slabs_handle;

/* First global row of every slab: row_starts[k] for k = 0..nslabs
 * (row_starts[nslabs] = ny); host only.  EINVAL if a slab would have fewer
 * than 3 rows. */
wblbe_status wblbe_slabs_rows(int32_t ny, int32_t nslabs, int32_t* row_starts);

/* Device workspace bytes for a split into nslabs slabs; 0 if invalid. */
size_t wblbe_slabs_workspace_bytes(const wblbe_params* params, int32_t nslabs);

/* Create a split lattice (workspace borrowed until destroy).  EINVAL on
 * bad parameters, scheme 4, too many slabs or a short/misaligned workspace
 * (ENOMEM when only short); ECUDA if its streams or events cannot be
 * created.  Synchronous (uploads the exchange table). */
wblbe_status wblbe_slabs_create(const wblbe_params* params, int32_t nslabs,
                                void* dev_workspace, size_t workspace_bytes,
                                void* cuda_stream, wblbe_slabs_handle* out);

/* As wblbe_init_rho: u = 0, f = f^eq(rho, 0); rho [ny][nx] float64. */
wblbe_status wblbe_slabs_init_rho(wblbe_slabs_handle h, const double* rho,
                                  int32_t rho_on_device);

/* Advance nsteps steps (every slab, then the ghost-row exchange). */
wblbe_status wblbe_slabs_step(wblbe_slabs_handle h, int64_t nsteps);

/* As wblbe_moments, for the whole lattice (fields [ny][nx], each may be
 * NULL; stats reduced over all slabs in a fixed order).  Synchronises. */
wblbe_status wblbe_slabs_moments(wblbe_slabs_handle h, double* rho, double* ux,
                                 double* uy, double* mu, int32_t out_on_device,
                                 wblbe_stats* stats);

/* The whole lattice's populations f_i(x, t) as [9][ny][nx] float64. */
wblbe_status wblbe_slabs_get_populations(wblbe_slabs_handle h, double* f,
                                         int32_t on_device);
int64_t wblbe_slabs_step_count(wblbe_slabs_handle h);
int64_t wblbe_slabs_kernel_launches(wblbe_slabs_handle h);
wblbe_status wblbe_slabs_destroy(wblbe_slabs_handle h);
const char* wblbe_slabs_last_error(wblbe_slabs_handle h);

/* ---- three dimensions: D3Q19, FP64 or FP32-shifted -------------------------
 * The paper's construction is written for D dimensions (Eq. mFeq, Eq. mF and
 * Eq. mFi, whose isotropic term carries D; Sec. V notes it carries over to
 * other LBE models).  These entry points run it, and the standard scheme, on
 * the D3Q19 lattice (D = 3, cs^2 = 1/3, weights 1/3, 1/18, 1/36) with the
 * isotropic central stencils grad(phi) = 3 sum_i w_i c_i phi(x + c_i),
 * lap(phi) = 6 sum_i w_i (phi(x + c_i) - phi(x)), periodic in x, y, z, in
 * float64 or float32-shifted storage (below).  Direction order (rest, axes,
 * edges in opposite pairs):
 *   c0 = (0,0,0); c1..c6 = (1,0,0) (-1,0,0) (0,1,0) (0,-1,0) (0,0,1) (0,0,-1);
 *   c7..c18 = (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0) (1,0,1) (-1,0,-1)
 *             (1,0,-1) (-1,0,1) (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1).
 * Scalar fields are [nz][ny][nx] float64 (x fastest); u is [3][nz][ny][nx];
 * populations [19][nz][ny][nx].  Conventions as for the 2D API.
 * WBLBE_FP32_SHIFTED stores float32 deviations g_i = f_i - s_i from the
 * scheme's rest equilibrium at rho_ref = rho_g (and the well-balanced rho0
 * vector), with float32 arithmetic and float64 reductions; in the
 * well-balanced scheme the rest population comes from the exact node mass
 * balance and is rounded stochastically, one draw per node from a hash of
 * the node and the step, as in 2D. */
typedef struct wblbe3_ctx* wblbe3_handle;

typedef struct {
  int32_t nx, ny, nz;              /* ny, nz <= 65535                      */
  double tau, kappa, beta, rho_l, rho_g;
  double rho0;                     /* Eq. mFeq; well-balanced scheme only  */
  int32_t scheme;                  /* WBLBE_STANDARD | WBLBE_WELL_BALANCED */
  int32_t precision;               /* WBLBE_FP64 | WBLBE_FP32_SHIFTED      */
} wblbe3_params;

/* Workspace bytes (0 on invalid parameters): two population buffers, the
 * density and chemical-potential fields, staging and reduction records. */
size_t wblbe3_workspace_bytes(const wblbe3_params* params);
wblbe_status wblbe3_create(const wblbe3_params* params, void* dev_workspace,
                           size_t workspace_bytes, void* cuda_stream,
                           wblbe3_handle* out);
/* u = 0, f = f^eq(rho, 0); rho [nz][ny][nx] on the host or device. */
wblbe_status wblbe3_init_rho(wblbe3_handle h, const double* rho,
                             int32_t rho_on_device);
/* Advance nsteps steps (three kernels per step; asynchronous). */
wblbe_status wblbe3_step(wblbe3_handle h, int64_t nsteps);
/* rho, u ([3][nz][ny][nx]), mu (each may be NULL) and the stats of the
 * current state.  Synchronises. */
wblbe_status wblbe3_moments(wblbe3_handle h, double* rho, double* u, double* mu,
                            int32_t out_on_device, wblbe_stats* stats);
wblbe_status wblbe3_get_populations(wblbe3_handle h, double* f, int32_t on_device);
int64_t wblbe3_step_count(wblbe3_handle h);
int64_t wblbe3_kernel_launches(wblbe3_handle h);
wblbe_status wblbe3_destroy(wblbe3_handle h);
const char* wblbe3_last_error(wblbe3_handle h);

/* ---- allocation-free statistics pass ------------------------------------
 * The paper has no counterpart of this entry point.  It serves callers that
 * cannot allocate device memory at all: hosts whose own allocator has
 * reserved the whole device and forbids cudaMalloc, and plug-ins or
 * callbacks that only ever receive buffers.  It computes, from
 * caller-held populations f ([9][ny][nx] float64 on the device, the layout of
 * wblbe_get_populations), the fields rho, ux, uy, mu ([ny][nx] float64 device
 * pointers, each may be NULL) and the stats (host pointer, may be NULL;
 * step and mass_drift_rel are returned as 0), exactly as wblbe_moments does
 * for a handle holding that state.  params->precision must be WBLBE_FP64.
 *
 * It allocates nothing and creates no handle: its only scratch is a fixed
 * array inside the library (16385 records of 6 float64, about 786 KB), which
 * every GPU that loads the library holds until the process exits.  Lattices
 * needing more than ceil(nx/32) * ceil(ny/8) = 16384 records (for example
 * 4096 x 4096 needs 65536; 1024 x 1024 needs 4096) are rejected with
 * WBLBE_ENOMEM.  The first call on a device looks up that device's address
 * of the array (cudaGetSymbolAddress).  All calls share the one array:
 * calls that overlap on the GPU (different streams, or different host
 * threads on one device) race and must be serialised by the caller.  Work is issued on cuda_stream (NULL =
 * legacy default stream); when stats is not NULL the call synchronises that
 * stream.  Errors: EINVAL (NULL params/f, invalid parameters, precision not
 * FP64), ENOMEM (lattice too large for the scratch), ECUDA.  The message of
 * the last failure on the calling thread is wblbe_noalloc_last_error(). */
wblbe_status wblbe_moments_noalloc(const wblbe_params* params, const double* f,
                                   double* rho, double* ux, double* uy,
                                   double* mu, wblbe_stats* stats,
                                   void* cuda_stream);
const char* wblbe_noalloc_last_error(void);

/* Measurement aid (no counterpart in the paper): the device's float64
 * fused multiply-add rate, the ceiling of the float64 step kernel, which is
 * bound by FP64 arithmetic rather than by memory traffic.  Launches
 * `blocks` CTAs of `threads` threads (a multiple of 32, at most 1024); each
 * thread runs 8 independent chains of `iters` fused multiply-adds and
 * writes one float64 to out (a device array of blocks * threads doubles,
 * owned by the caller).  One launch performs blocks * threads * iters * 8
 * FMAs (2 flops each).  Asynchronous on cuda_stream; the caller times it.
 * EINVAL on bad arguments, ECUDA if the launch fails. */
wblbe_status wblbe_probe_fp64_fma(double* out, int32_t blocks, int32_t threads,
                                  int32_t iters, void* cuda_stream);

/* Measurement aid (no counterpart in the paper): the reciprocal 1/rho that
 * the float64 update uses for u = (sum_i c_i f_i + F/2) / rho (Eq. rhoU),
 * evaluated on n device values x: seed[i] = the hardware approximation it
 * starts from, refined[i] = the refined reciprocal the kernels use (either
 * output may be NULL, not both).  Device arrays of n doubles, owned by the
 * caller; asynchronous on cuda_stream.  EINVAL on bad arguments. */
wblbe_status wblbe_probe_reciprocal(const double* x, double* seed, double* refined,
                                    int64_t n, void* cuda_stream);

/* Debugging aid (no counterpart in the paper).  Compute-sanitizer is not
 * available where this library is tested, so a build with
 * -DWBLBE_DEBUG_BOUNDS checks every global access of the step, moments and
 * batched kernels (and the shared-memory slots they compute at run time)
 * before making it; an access out of its buffer is skipped and counted.
 * Returns that count on the current device (reset != 0 clears it),
 * 0xFFFFFFFF in a library built without the checks, 0xFFFFFFFE if the count
 * could not be read. */
unsigned int wblbe_debug_bounds_errors(int32_t reset);

#ifdef __cplusplus
}
#endif

#endif /* WBLBE_H */
