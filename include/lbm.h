/*
 * lbm.h - C ABI of the GB300 two-component MRT pseudopotential lattice
 * Boltzmann solver with the corrected open boundaries of arxiv 2512.12934.
 *
 * Conventions (every entry point):
 *  - Plain C types only; no C++ or framework types cross this boundary.
 *  - The library owns all device state it allocates.  The caller owns every
 *    host buffer it passes; the library never keeps a host pointer past the
 *    call that received it.
 *  - Fields are row-major with x fastest: a scalar field is [nz][ny][nx]
 *    (nz = 1 in 2D); a per-component field is [2][nz][ny][nx]; a vector
 *    field is [dim][nz][ny][nx] with dim = 2 (D2Q9) or 3 (D3Q19).
 *  - Work is enqueued on the CUDA stream given at creation (NULL = the
 *    legacy default stream).  Calls that return data synchronise that
 *    stream.  No C++ exception crosses the boundary; a numerical failure
 *    is a status code, never a device trap.
 *  - One context must not be used from two threads at once; separate
 *    contexts are independent.
 *  - A failing call returns a non-zero lbm_status and records a message
 *    readable with lbm_last_error().
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_ERR_INVALID_ARG = 1, /* rejected before any device work */
    LBM_ERR_CUDA = 2,        /* a CUDA runtime call failed */
    LBM_ERR_OOM = 3,         /* device or host allocation failed */
    LBM_ERR_DIVERGED = 4,    /* a non-finite density or velocity appeared */
    LBM_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
    LBM_ERR_UNSUPPORTED = 6, /* valid request this library does not implement */
    LBM_ERR_IO = 7           /* checkpoint file could not be read/written */
} lbm_status;

enum { LBM_D2Q9 = 0, LBM_D3Q19 = 1 };

/* Arithmetic / storage of the populations.  FP32: f stored and computed in
 * float.  FP32_FP16STORE: f stored as half deviations from w_i * rho_ref,
 * rho_ref being the half-rounded density of the node that pulls the value in
 * the next step (per node and component, stored alongside: 80 B per node and
 * step instead of 144), computed in float.  FP64: stored and computed in
 * double (diagnostic). */
enum { LBM_FP32 = 0, LBM_FP32_FP16STORE = 1, LBM_FP64 = 2 };

enum { LBM_INLET_VELOCITY = 1, LBM_OUTLET_CONVECTIVE = 2 };
enum { LBM_XMIN = 0, LBM_XMAX = 1, LBM_YMIN = 2, LBM_YMAX = 3, LBM_ZMIN = 4, LBM_ZMAX = 5 };

/* s_eps choice: own viscosity of each component (the uncorrected scheme) or
 * the largest viscosity of the two phases (Sec. III A of the paper). */
enum { LBM_SEPS_OWN_NU = 0, LBM_SEPS_MAX_NU = 1 };

/* Step schedules (lbm_set_schedule, lbm_batch_set_schedule). */
enum { LBM_SCHEDULE_GRAPHS = 0, LBM_SCHEDULE_PERSISTENT = 1, LBM_SCHEDULE_GRAPHS_EARLY = 2 };

typedef struct lbm_ctx lbm_ctx; /* opaque, library-owned */

/* Lattice and grid.  nz = 1 for D2Q9.  Every non-periodic extent must be
 * >= 5 (the interaction stencil of Eq. 10 reaches two nodes). */
typedef struct {
    int lattice;     /* LBM_D2Q9 or LBM_D3Q19 */
    int nx, ny, nz;
    int periodic[3]; /* non-zero: that axis wraps (App. B, Eq. B2) */
} lbm_grid;

/* Physical parameters (Sec. II A).
 *  G12        fluid-fluid strength of Eq. 10 (weights as printed).
 *  Gw[k]      adhesion strength of Eq. 11 for component k (constant).
 *  nu[k]      kinematic viscosity; s_nu,k = 1/(3 nu_k + 1/2) (Eq. 5);
 *             must give 0 < s_nu,k < 2.
 *  s_e        rate of the energy moment; <= 0 selects s_e,k = s_nu,k.
 *  s_q        rate of both heat-flux moments (Eq. 4); <= 0 selects 1.2.
 *  s_eps_mode LBM_SEPS_MAX_NU (paper) or LBM_SEPS_OWN_NU.
 *  body_force body-force density, shared between components by rho_k/rho.
 *  precision  LBM_FP32, LBM_FP32_FP16STORE or LBM_FP64.
 *  rho0_store reserved (ignored: FP16 storage references per-node densities). */
typedef struct {
    double G12;
    double Gw[2];
    double nu[2];
    double s_e;
    double s_q;
    int s_eps_mode;
    double body_force[3];
    int precision;
    double rho0_store;
} lbm_params;

/* One open face (Sec. II B).  The face is the whole grid side `side`,
 * restricted to the inclusive extent [lo, hi] along its tangential axes
 * (index 0 = the first tangential axis in x, y, z order; index 1 is used in
 * 3D only).  Solid nodes inside the extent are skipped.
 *  kind = LBM_INLET_VELOCITY: NEQ extrapolation of the unknown populations
 *    (Eqs. 13, 14) followed, when alpha_correction != 0, by the alpha
 *    correction (Eqs. 15-19).  u_profile (host, may be NULL = 0) holds the
 *    inflow speed along the inward normal at each face position, row-major
 *    over the extent; rho_in[k] are the prescribed component densities.
 *  kind = LBM_OUTLET_CONVECTIVE: convective outflow (Eqs. 20, 21); when
 *    chi_correction != 0 the outlet normal velocity is rescaled by the
 *    mass-flux ratio chi (Eqs. 22, 23).
 * At most one outlet face.  The inward neighbour of every face node must be
 * an ordinary fluid node.  A face may not lie on a periodic axis. */
typedef struct {
    int kind;
    int side;
    int lo[2], hi[2];
    const double* u_profile;
    double rho_in[2];
    int alpha_correction;
    int chi_correction;
    const double* rho_profile;
} lbm_open_bc;

/* Diagnostics (FP64 reductions on the device).
 *  mass[k]   sum of rho_k over the fluid nodes (post-collision state);
 *  lambda    outlet coefficient of Eq. 21 the next step will use;
 *  chi       outlet correction of Eq. 23 the next step will use;
 *  q_in      inlet mass flux sum (rho_1+rho_2) u.n_in of the last step;
 *  q_out     the same at the column x_{N-1} next to the outlet;
 *  max_speed largest |u^eq| of the last reported macroscopic fields;
 *  step      number of completed time steps;
 *  launches  number of kernels this context has launched;
 *  status    LBM_OK or LBM_ERR_DIVERGED. */
typedef struct {
    double mass[2];
    double lambda, chi, q_in, q_out;
    double max_speed;
    int64_t step;
    int64_t launches;
    int status;
} lbm_diag;

/* Create a solver (Sec. II; call stack of one time step below).
 *  solid     host [nz][ny][nx] bytes, non-zero = solid node; NULL = none.
 *  rho_init  host [2][nz][ny][nx] initial component densities.
 *  u_init    host [dim][nz][ny][nx] initial common velocity; NULL = 0.
 *  cuda_stream  a cudaStream_t (NULL = legacy default stream).
 * The initial populations are the equilibria of Eq. 6 at (rho_k, u).
 * Returns LBM_ERR_INVALID_ARG (nothing allocated) for an invalid grid,
 * rates outside (0, 2), a bad face, or a NULL required pointer. */
lbm_status lbm_create(const lbm_grid* grid, const lbm_params* params,
                      const lbm_open_bc* bcs, int nbc, const uint8_t* solid,
                      const double* rho_init, const double* u_init,
                      void* cuda_stream, lbm_ctx** out);

/* Restart the context from new initial fields on the same grid, faces and
 * parameters (host rho_init [2][nz][ny][nx], u_init [dim][nz][ny][nx] or
 * NULL): populations become the equilibria of Eq. 6, the open-boundary
 * state is cleared (lambda = 0, chi = 1), the step counter returns to 0. */
lbm_status lbm_reset(lbm_ctx* ctx, const double* rho_init, const double* u_init);

/* Enqueue nsteps time steps (nsteps >= 0) on the context's stream.  A step
 * performs, fused per tile of nodes: pull streaming (Eq. 2) with halfway
 * bounce-back (Eq. B1) and periodic wrap (Eq. B2); inlet reconstruction
 * (Eqs. 13-19); convective outlet (Eqs. 20, 21); densities and
 * pseudopotentials with ghost mirrors (Eqs. 24, 25); forces (Eqs. 10, 11);
 * common velocity (Eqs. 7, 8) with the outlet rescaled by chi (Eq. 22); MRT
 * collision with forcing (Eqs. 1, 3-6, 9); and the FP64 flux reductions that
 * give lambda and chi for the next step (Eqs. 21, 23).  D2Q9 launches per
 * step (graph schedule): one for the general tiles (those that see an open
 * face) and one for the other tiles, plus one for the column-marching runs
 * under tile variant 4 (FP32); the persistent schedule runs up to 1024
 * steps per launch.  D3Q19: five launches per step (pulls, face pulls,
 * collision, outlet, reduction).  Returns without waiting for the GPU;
 * launch errors are reported at once, divergence (LBM_ERR_DIVERGED) or a
 * bounded device wait that ran out (LBM_ERR_TIMEOUT) by the next call that
 * synchronises (lbm_sync, lbm_get_*). */
lbm_status lbm_step(lbm_ctx* ctx, int64_t nsteps);

/* Wait for the context's stream; LBM_ERR_DIVERGED if a non-finite density
 * or velocity was produced since creation (or the last lbm_reset),
 * LBM_ERR_TIMEOUT if a bounded device wait ran out. */
lbm_status lbm_sync(lbm_ctx* ctx);

/* Macroscopic fields used by the most recent collision (after creation:
 * the initial fields): rho [2][nz][ny][nx] and u^eq [dim][nz][ny][nx], as
 * float.  dst_is_device != 0: both pointers are device memory on the
 * context's device (e.g. a torch CUDA tensor's data_ptr); otherwise host.
 * Solid nodes read 0. */
lbm_status lbm_get_macros(lbm_ctx* ctx, float* rho, float* u, int dst_is_device);

/* The same fields as double, host memory only. */
lbm_status lbm_get_macros_f64(lbm_ctx* ctx, double* rho, double* u);

/* Post-collision populations [2][Q][nz][ny][nx] (host, double), Q = 9 or 19,
 * in the velocity order of the lattice (D2Q9: e_0..e_8 as in Eq. 13/20). */
lbm_status lbm_get_populations(lbm_ctx* ctx, double* f);

/* Overwrite the post-collision populations (host, double, same layout). */
lbm_status lbm_set_populations(lbm_ctx* ctx, const double* f);

/* FP64 diagnostics; synchronises. */
lbm_status lbm_get_diagnostics(lbm_ctx* ctx, lbm_diag* out);

/* Checkpoint: populations, open-boundary state, lambda, chi and the step
 * counter, so that n steps = k steps + save + load + (n-k) steps bit for bit. */
lbm_status lbm_save(lbm_ctx* ctx, const char* path);
lbm_status lbm_load(lbm_ctx* ctx, const char* path);

/* Kernel timing.  every > 0: from now on every `every`-th step kernel is
 * launched on its own between a pair of CUDA events recorded on the
 * context's stream (at most 4096 samples are kept); every = 0 turns
 * sampling off.  Either call clears the samples.  lbm_kernel_time
 * synchronises and returns the mean device duration of the sampled step
 * launches in milliseconds and how many were sampled. */
lbm_status lbm_enable_kernel_timing(lbm_ctx* ctx, int every);
lbm_status lbm_kernel_time(lbm_ctx* ctx, double* mean_ms, int64_t* samples);

/* The same samples split by launch: the fast tile list (interior and edge
 * tiles) and the general tile list (tiles that see an open face), each a
 * mean device duration in milliseconds (0 for an empty list). */
lbm_status lbm_kernel_time_split(lbm_ctx* ctx, double* fast_ms, double* general_ms, int64_t* samples);

/* Tile shape of the fused step kernel: variant in [0, lbm_num_tile_variants()),
 * 0: 32x8, 1: 32x4, 2: 64x4, 3: 32x16 nodes per CTA (default: 1 below 2^22
 * nodes, else 0).  Bit-identical results on grids without open faces; with
 * open faces the FP64 flux partials are grouped per tile, so chi may differ
 * in its last bit.  Variant 4 tiles like variant 0 and, for FP32 storage,
 * runs the interior tiles (those whose pulls and interaction stencil stay
 * inside the grid and away from open faces) through the column-marching
 * kernel: one CTA per run of up to 64 tiles of a tile column, one TMA bulk
 * copy of all 18 population planes per 8 rows, pulls from shared memory.
 * Same method; results agree with variant 0 to FP32 rounding.  Other
 * precisions run variant 4 exactly as variant 0.  Batches and the
 * persistent schedule run variant 4 members as variant 0. */
lbm_status lbm_set_tile_variant(lbm_ctx* ctx, int variant);
int lbm_num_tile_variants(void);

/* Current tiling: variant, number of tiles in the fast and general lists and
 * the fluid nodes each list owns (every fluid node belongs to exactly one). */
lbm_status lbm_tile_stats(lbm_ctx* ctx, int* variant, int* fast_tiles, int* general_tiles,
                          int64_t* fast_nodes, int64_t* general_nodes);

/* Step-replay mode: use_graphs != 0 (the default) replays runs of steps
 * from captured CUDA graphs (two launches per graph node pair, captured on
 * first use); 0 launches every step individually.  Results are identical. */
lbm_status lbm_set_graph_mode(lbm_ctx* ctx, int use_graphs);

/* Moving wall beyond a closed y edge (side LBM_YMIN: the halfway wall at
 * y = -1/2, LBM_YMAX: at y = ny - 1/2) with x-velocity ux (|ux| <= 0.2;
 * 0 = at rest, the default).  The paper shears droplets between plates
 * moving in opposite directions (Taylor deformation, Sec. III A) without
 * giving the wall scheme; here a population reflected at the wall gains
 * 2 w_i rho_k (e_i . u_w) / c_s^2, rho_k the node's own density before
 * streaming (halfway bounce-back with the wall's momentum), which keeps
 * plane Couette flow exact.  Needs a non-periodic y axis without an open
 * face on that side; FP32 and FP64 storage.  Applies from the next step
 * (a running batch picks it up when rebuilt).  Waits for the stream. */
lbm_status lbm_set_wall_velocity(lbm_ctx* ctx, int side, double ux);

/* Wettability, Eq. 12.  The paper makes the adhesion coefficient of Eq. 11
 * depend on a phase quantity rho^e through a threshold delta and two
 * functions g1, g2 that it does not define (they come from its ref. [42]).
 * delta in (0, 1] switches on this library's reading: one coefficient for
 * both components, G_w(rho^e) with rho^e = (rho_1 - rho_2)/(rho_1 + rho_2)
 * at the node: Gw[0] (lbm_params) where rho^e > delta, Gw[1] where
 * rho^e < -delta, and the linear pieces g1 = Gw[0] rho^e/delta on
 * (0, delta], g2 = -Gw[1] rho^e/delta on (-delta, 0] between them (zero
 * on the interface itself).  In either pure phase the dominant component
 * then feels exactly its constant coefficient; only the contact-line region
 * changes.  delta <= 0 (the default): each component keeps its constant
 * Gw[k].  Applies from the next step.  Waits for the context's stream. */
lbm_status lbm_set_wetting(lbm_ctx* ctx, double delta);

/* Timing of chi, the outlet mass-flux correction (Eqs. 22, 23).
 *  same_step = 0 (default): chi of a step comes from the previous step's
 *    inlet and outlet fluxes (one-step lag), so each step needs no grid-wide
 *    sum before its collisions.
 *  same_step = 1: chi comes from the step's own fluxes, as Eq. 23 is printed
 *    (t + dt): after the general tiles of each step one more launch sums the
 *    step's FP64 flux partials, sets the outlet nodes' normal velocity
 *    (Eq. 22) and collides them.  lambda (Eq. 21) stays lagged in both: Eq.
 *    20 needs it before the step's velocities exist.
 * No effect without an outlet carrying the chi correction.  FP32 and FP64
 * storage, graph schedule, contexts outside batches; LBM_ERR_UNSUPPORTED
 * otherwise.  Waits for the context's stream. */
lbm_status lbm_set_chi_timing(lbm_ctx* ctx, int same_step);

/* Schedule of lbm_step for this context: LBM_SCHEDULE_GRAPHS (default),
 * LBM_SCHEDULE_GRAPHS_EARLY or LBM_SCHEDULE_PERSISTENT (FP32 storage only);
 * see lbm_batch_set_schedule, of which this is the one-member case.  Under
 * the persistent schedule lbm_sync also reports LBM_ERR_TIMEOUT, and
 * lbm_enable_kernel_timing takes no samples.  Waits for the context's
 * stream first.  2D contexts only (LBM_ERR_UNSUPPORTED for D3Q19). */
lbm_status lbm_set_schedule(lbm_ctx* ctx, int schedule);

/* The context's schedule, and in *early_in_use whether its instantiated
 * step graphs launch early (1) or, the driver having refused the
 * programmatic edges, are plain graphs (0; also before the first graph is
 * built, and always for D3Q19 contexts, which report LBM_SCHEDULE_GRAPHS).
 * Never blocks. */
lbm_status lbm_get_schedule(lbm_ctx* ctx, int* schedule, int* early_in_use);

/* FP64 mass of each component of caller-owned D2Q9 populations, for callers
 * that cannot allocate device memory (a process whose device memory is all
 * owned by another allocator or arena).  The paper has no counterpart: this
 * is the lbm_get_diagnostics mass tally without a context and without any
 * cudaMalloc.
 *  f         device populations [2][9][ny][pitch], float (precision =
 *            LBM_FP32) or double (LBM_FP64); read only.
 *  solid     device mask [ny][pitch], non-zero = solid (skipped); may be NULL.
 *  mass      device output, 2 doubles (sum over fluid nodes of sum_i f_i).
 *  cuda_stream  stream to enqueue on (NULL = legacy default stream).
 * The per-row partial sums live in one fixed device array of 65536 rows x 2
 * doubles (1 MiB) that every GPU loading this library keeps until process
 * exit; ny > 65536 is rejected with LBM_ERR_INVALID_ARG.  Every call on a
 * device reuses that array, so calls that overlap on the GPU (concurrent
 * streams or host threads) race and give wrong sums; serialise them.  Each
 * call outside a stream capture resolves the array's device address in the
 * current context (so the address stays valid across cudaDeviceReset); a
 * call inside a capture reuses the address resolved by the last call on
 * that device outside a capture, so make one call on each device before
 * capturing (a capture with no earlier call fails with
 * LBM_ERR_INVALID_ARG), and do not reset the device between that call and
 * the capture.  If a CUDA error from earlier work is pending on the calling
 * thread the call launches nothing and returns LBM_ERR_CUDA, leaving that
 * error in place for its owner.
 * Returns without waiting; the result is ready when the stream reaches it. */
lbm_status lbm_mass_noalloc(const void* f, int precision, int nx, int ny, int pitch,
                            const uint8_t* solid, double* mass, void* cuda_stream);

/* ---- Batched ensembles (many independent instances, one launch per tile
 * list per step for all of them) ----------------------------------------
 * The paper runs one case at a time; batching is how many parameter points
 * (uneven grids, faces and parameters) share the GPU.  A batch refers to
 * existing contexts (the members, created with lbm_create, all of one
 * precision); the caller keeps owning them and may still read them between
 * batch steps (lbm_get_macros, lbm_get_diagnostics, ...).  Every member takes
 * the batch's tile variant.  A batch step advances every member by one time
 * step with exactly the arithmetic of lbm_step on that member alone. */
typedef struct lbm_batch lbm_batch;

/* members: n >= 1 distinct contexts of one precision; cuda_stream: the stream
 * batch work is enqueued on (NULL = legacy default stream). */
lbm_status lbm_batch_create(lbm_ctx* const* members, int n, void* cuda_stream, lbm_batch** out);

/* Enqueue nsteps steps of every member (runs of 32 steps replay captured
 * CUDA graphs); members' macroscopic fields are written by the last one. */
lbm_status lbm_batch_step(lbm_batch* b, int64_t nsteps);

/* Wait for the batch stream; LBM_ERR_DIVERGED if any member diverged,
 * LBM_ERR_TIMEOUT if a persistent launch's barrier wait ran out. */
lbm_status lbm_batch_sync(lbm_batch* b);

/* Re-tile every member with `variant` (see lbm_set_tile_variant). */
lbm_status lbm_batch_set_tile_variant(lbm_batch* b, int variant);

/* Autotuner: times `steps` batch steps of every tile variant from the
 * current state (restored afterwards, so the run is unchanged) and keeps the
 * fastest.  variant: the choice; ms_per_step (may be NULL): its time. */
lbm_status lbm_batch_autotune(lbm_batch* b, int steps, int* variant, double* ms_per_step);

/* The same for a single context (tile variants 0-3; FP32 contexts also time
 * the column-marching variant 4 on the context itself). */
lbm_status lbm_autotune(lbm_ctx* ctx, int steps, int* variant, double* ms_per_step);

/* Tile variant, number of tiles in the batch's fast and general lists and
 * kernel launches issued by the batch so far. */
lbm_status lbm_batch_info(lbm_batch* b, int* variant, int* fast_tiles, int* general_tiles, int64_t* launches);

/* CUDA-graph replay on (default) or off for batch steps. */
lbm_status lbm_batch_set_graph_mode(lbm_batch* b, int use_graphs);

/* How a batch step call runs on the GPU.
 *  LBM_SCHEDULE_GRAPHS (default): per time step, one launch for the fast
 *    tile list and one for the general list, replayed from captured CUDA
 *    graphs in runs of 32 steps.
 *  LBM_SCHEDULE_PERSISTENT (FP32 storage only): one cooperative launch per
 *    run of up to 1024 steps.  Its CTAs (as many as fit on the GPU at once,
 *    at most one per tile) walk the concatenated tile descriptors of all
 *    members in every step and meet at a grid-wide barrier between steps;
 *    each wait at that barrier is bounded (about one second of SM clock by
 *    default), and a wait that runs out ends the launch: lbm_batch_sync then
 *    returns LBM_ERR_TIMEOUT, after which the members' states are undefined
 *    (lbm_reset them before going on).  General tiles stage serially on the
 *    tile's node threads.  Results equal the graph schedule's to the FP32
 *    parity tolerance (not bit for bit: the general tiles' staging is
 *    compiled separately).
 *  LBM_SCHEDULE_GRAPHS_EARLY: the graph schedule with early launches.  In
 *    the captured graphs every dependency between two kernels becomes a
 *    programmatic one that lets the later kernel launch as soon as all CTAs
 *    of the earlier one have started; each step kernel waits on the device
 *    (griddepcontrol.wait, its first instruction) until the grids it
 *    depends on have completed and their writes are visible.  Every memory
 *    access keeps the plain graph's order, so results are bit-identical to
 *    LBM_SCHEDULE_GRAPHS; the launch latency between steps is hidden behind
 *    the previous step.  If the driver refuses the programmatic edges, the
 *    plain graphs are used (lbm_batch_get_schedule reports which).
 * The schedule applies from the next lbm_batch_step; switching between the
 * two graph forms waits for the batch's stream and drops its graphs. */
lbm_status lbm_batch_set_schedule(lbm_batch* b, int schedule);

/* The batch's schedule and whether its step graphs launch early (see
 * lbm_get_schedule).  Never blocks. */
lbm_status lbm_batch_get_schedule(lbm_batch* b, int* schedule, int* early_in_use);

/* CTAs of the batch's last persistent launch (0 before the first). */
lbm_status lbm_batch_persistent_grid(lbm_batch* b, int* ctas);

/* Failure-detection test hook (host-side injection; no device fault).  From
 * the next persistent launch on, every grid barrier waits for extra_arrivals
 * more CTAs than the grid has, so a barrier with extra_arrivals > 0 can never
 * complete and its waits run out after spin_limit_cycles SM clock cycles
 * (<= 0: the default budget); the launch then ends and lbm_batch_sync
 * reports LBM_ERR_TIMEOUT.  extra_arrivals = 0 restores normal operation.
 * Waits for the batch stream first. */
lbm_status lbm_batch_inject_barrier_fault(lbm_batch* b, int extra_arrivals, int64_t spin_limit_cycles);

/* Release the batch (not its members).  NULL is ignored. */
void lbm_batch_destroy(lbm_batch* b);

/* Message of the batch's last failure (b == NULL: the thread's last). */
const char* lbm_batch_last_error(const lbm_batch* b);

/* ---- Surrogate MLP ensemble ---------------------------------------------
 * The paper has no counterpart: it reports droplet sizes and generation
 * periods of T-junction and co-flow devices as functions of Ca, the flow-rate
 * ratio, the viscosity ratio and the width ratio (Sec. 4, Figs. 10-11); the
 * surrogate learns that map from runs of this solver.
 * Network of one member: x (4) -> 128 -> 128 -> 128 -> y (2), GELU
 * (z * Phi(z), the erf form) after each hidden layer, FP32 arithmetic
 * (inference by default on the tensor cores, as FP32-accurate split
 * products: lbm_mlp_set_infer_path).
 * Loss: mean squared error over the batch and both outputs.  Optimiser: Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).
 * Parameters of one member, flat float order (row-major, output index
 * first): W1[128][4], b1[128], W2[128][128], b2[128], W3[128][128], b3[128],
 * W4[2][128], b4[2]; lbm_mlp_num_params() floats.  All members lie back to
 * back: [members][num_params].
 * Host arrays: X [n][4] inputs, T [n][2] targets, row-major.  Every call
 * waits for its own work.  Per-call device buffers come from a workspace
 * the ensemble owns, grown (never shrunk) to the largest request so far and
 * released by lbm_mlp_destroy.  One lbm_mlp is not thread-safe. */
typedef struct lbm_mlp lbm_mlp;

int64_t lbm_mlp_num_params(void);

/* members in [1, 64]; weights uniform in +-1/sqrt(fan_in) from a splitmix64
 * stream seeded per member, biases 0; Adam moments 0. */
lbm_status lbm_mlp_create(int members, uint64_t seed, void* cuda_stream, lbm_mlp** out);

/* Replace all members' parameters (host, members*num_params floats); resets
 * the Adam moments and step count. */
lbm_status lbm_mlp_set_params(lbm_mlp* m, const float* params);
/* Copy all members' parameters out (host, members*num_params floats). */
lbm_status lbm_mlp_get_params(lbm_mlp* m, float* params);

/* Every member's output on n inputs: Y [members][n][2] (host).  On the
 * tensor-core path a bounded device wait that ran out returns
 * LBM_ERR_TIMEOUT (outputs undefined; the ensemble stays usable). */
lbm_status lbm_mlp_forward(lbm_mlp* m, const float* X, int n, float* Y);

/* Full-batch gradient of every member's loss on (X, T): grad
 * [members][num_params] (host).  Parameters are not changed. */
lbm_status lbm_mlp_gradient(lbm_mlp* m, const float* X, const float* T, int n, float* grad);

/* Adam training: `epochs` passes over (X, T), each a splitmix64
 * Fisher-Yates shuffle (seeded by shuffle_seed, continued across epochs)
 * cut into minibatches of `batch` rows (a ragged tail is dropped); every
 * member sees the same minibatches.  batch > n is clamped to n. */
lbm_status lbm_mlp_train(lbm_mlp* m, const float* X, const float* T, int n, int epochs, int batch, double lr,
                         uint64_t shuffle_seed);

/* Ensemble prediction on n inputs: mean [n][2] and spread [n], the largest
 * over the two outputs of (population std over members) / |mean|.
 * dst_is_device != 0: X, mean and spread are device pointers on the
 * library's device (enqueued on the stream, still waited for). */
lbm_status lbm_mlp_predict(lbm_mlp* m, const float* X, int n, float* mean, float* spread, int dst_is_device);

/* Inference paths of lbm_mlp_forward and lbm_mlp_predict (training always
 * runs on the FP32 pipes).
 *  LBM_MLP_INFER_SIMT: FP32 FMAs, 128-sample tiles with 8x8 register blocks.
 *  LBM_MLP_INFER_TENSOR (default): the two 128x128 hidden layers on the tcgen05
 *    tensor cores as three accumulated products, tf32(A).tf32(W) +
 *    (A - tf32(A)).tf32(W) + bf16(A).bf16(W - tf32(W)), which keeps FP32-level
 *    error (below 2^-20 of |A||W| per product); layers 1 and 4, biases and
 *    GELU on the FP32 pipes.  Results differ from the SIMT path in the last
 *    bits (another summation order).
 * Waits for the ensemble's stream. */
enum { LBM_MLP_INFER_SIMT = 0, LBM_MLP_INFER_TENSOR = 1 };
lbm_status lbm_mlp_set_infer_path(lbm_mlp* m, int path);

/* Longest wait, in SM clock cycles, of the tensor-core inference kernel on
 * its weight copy and on its MMAs (0: the default, about a second).  A wait
 * that runs out ends the call with LBM_ERR_TIMEOUT; the kernel lets its own
 * weight copy land (default limit) and frees its tensor memory before it
 * leaves, so the ensemble stays usable.  Small limits exist to exercise
 * that path.  Waits for the ensemble's stream. */
lbm_status lbm_mlp_set_wait_limit(lbm_mlp* m, long long cycles);

/* Release the ensemble.  NULL is ignored. */
void lbm_mlp_destroy(lbm_mlp* m);

/* Message of the ensemble's last failure (m == NULL: the thread's last). */
const char* lbm_mlp_last_error(const lbm_mlp* m);

/* Release all device memory of the context.  NULL is ignored. */
void lbm_destroy(lbm_ctx* ctx);

/* Message of the last failure on ctx (ctx == NULL: the calling thread's last
 * failure outside a context, e.g. in lbm_create).  Never NULL. */
const char* lbm_last_error(const lbm_ctx* ctx);

/* Library version string. */
const char* lbm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
