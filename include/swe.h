/*
 * libswe — one time step of the combined Lagrangian-Euler (CSPH-TVD)
 * shallow-water scheme on a regular grid, on one NVIDIA GB300 (sm_103a).
 *
 * The method: Dyakonova, Khoperskov & Khrapov, "Numerical Model of Shallow
 * Water: the Use of NVIDIA CUDA Graphics Processors" (arXiv 1705.00614).
 * The state solves the Saint-Venant equations, Eqs. 1-3, with the force
 * terms of Eq. 4; a step is the four-stage scheme of Sec. 2.3 (Fig. 2),
 * computed by the paper's kernels K2-K8 (Sec. 3): forces, CFL time step,
 * Lagrangian predictor and corrector, Eulerian TVD face fluxes, final update.
 *
 * Conventions shared by every entry point
 *  - Every function returns a swe_status (0 = SWE_OK, negative = error) except
 *    swe_destroy and the string functions.  No C++ exception crosses the ABI.
 *    On error, swe_last_error() returns a message for the calling thread.
 *  - Host arrays are row-major [ny][nx] (x fastest), FP64, owned by the
 *    caller and only read or written during the call (they are copied).
 *    Cell (i, j) has centre ((i + 1/2) dx, (j + 1/2) dx).
 *  - A context owns all device memory it uses (allocated in swe_create and,
 *    for the staging buffer of host copies, at the first host copy) and
 *    frees it in swe_destroy.  Device pointers returned by
 *    swe_get_device_ptrs stay owned by the context.
 *  - A context is bound to one CUDA stream: swe_params.cuda_stream, or, when
 *    that is NULL, a non-blocking stream the context creates and destroys
 *    (the legacy default stream cannot hold the CUDA graphs swe_step uses).
 *    A context is not thread safe.  Calls that return data to the host
 *    synchronise that stream; the others only enqueue work.
 *  - Depth H (m), momentum Q = H U (m^2/s, the paper's HV of K8), bed b (m).
 */
#ifndef SWE_H
#define SWE_H

#include <stdint.h>

#if defined(__GNUC__)
#define SWE_API __attribute__((visibility("default")))
#else
#define SWE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct swe_ctx swe_ctx; /* opaque, owned by the library */

typedef enum {
    SWE_OK = 0,
    SWE_ERR_ARG = -1,            /* invalid argument; nothing was changed */
    SWE_ERR_CUDA = -2,           /* a CUDA call failed; see swe_last_error() */
    SWE_ERR_OOM = -3,            /* device or host allocation failed */
    SWE_ERR_NONFINITE = -4,      /* a NaN/Inf entered the state or the speeds */
    SWE_ERR_DT = -5,             /* time step not positive (t_end already reached) */
    SWE_ERR_DEVICE_TIMEOUT = -6, /* a bounded device wait ran out; the step is invalid */
    SWE_ERR_STATE = -7           /* call out of order (e.g. no state set yet) */
} swe_status;

enum { SWE_F32 = 0, SWE_F64 = 1 };           /* arithmetic and storage type */
enum { SWE_FUSED = 0, SWE_STAGED = 1 };      /* kernel organisation */

/* Parameters of one grid: the physical constants of Eqs. 1-4 and the
 * numerical ones of Sec. 2.3.  Zero-initialise and set what you need;
 * swe_params_default fills the usual values. */
typedef struct {
    int32_t nx, ny;        /* cells along x and y, each >= 1 */
    int32_t precision;     /* SWE_F32 or SWE_F64 */
    int32_t mode;          /* SWE_FUSED (one tiled kernel per step) or
                              SWE_STAGED (one kernel per stage, keeps every
                              intermediate in device memory) */
    double dx;             /* h = dx = dy (m), Sec. 2.2 */
    double g;              /* gravitational acceleration (m/s^2) */
    double cfl;            /* Courant number K, 0 < K < 1 (Fig. 2) */
    double eps_dry;        /* a cell is wet when H > eps_dry (the Eps of K8) */
    double dt_max;         /* upper bound of the time step (s) */
    double dt_fixed;       /* > 0: every step uses this tau instead of the CFL */
    double nu;             /* kinematic turbulent viscosity (m^2/s), Eq. 4 */
    double coriolis_f;     /* 2 Omega sin(latitude) (1/s), Eq. 4 */
    double wind_x, wind_y; /* wind velocity W (m/s), Eq. 4 */
    double c_a;            /* wind drag coefficient C_a, Eq. 4 */
    double rho_air_over_rho; /* rho_a / rho, Eq. 4 */
    void* cuda_stream;     /* cudaStream_t to run on; borrowed, may be NULL */
    int32_t tile_w;        /* fused mode: output columns per CTA (0 = auto) */
    int32_t seg_h;         /* fused mode: output rows per CTA (0 = auto: a launch-cost model, at most 256 with skip_dry) */
    int32_t skip_dry;      /* fused mode, 0 or 1: skip dry tiles (the wet-block
                              test of the paper's kernel K1, Sec. 3).  A work
                              item whose window (its cells and the 6-cell ring
                              a step reads) holds no wet cell and no source
                              cell is not computed: its cells keep H and get
                              Q = 0, bitwise what the full step computes for
                              them.  Wetness is kept per 32 x 16-cell block as
                              the last step at which the block held a wet
                              cell.  Never applied to swe_step_closed.
                              Off by default (throughput then does not depend
                              on the wet fraction). */
    int32_t ghost_ring;    /* fused mode, 0, 1 or 2: 0 = the SWE_PAD cells around
                              the grid are reflective walls; 1 = they are ghost
                              cells whose terrain the caller sets with
                              swe_set_terrain_ext and whose state a nest
                              (swe_nest_*) fills from a coarser grid before
                              every step (a ghost cell that is never filled is
                              dry ground, through which water can leave);
                              2 = open boundary: before every step each ghost
                              cell whose bed is below 1e29 takes the state of
                              the nearest interior cell (zero gradient), so
                              flow and waves leave the grid; ghosts with a bed
                              of 1e29 or more stay walls (set the ring terrain,
                              e.g. edge-extended, with swe_set_terrain_ext).
                              With CFL steps the signal speed then covers the
                              filled ring too (the padded extent stepped as
                              one grid).  After every fill the stored forces
                              of the ring band are recomputed.  Not in
                              batches (swe_batch_create refuses them). */
    /* Distributed sources of Eq. 1 on every non-wall cell, m/s, >= 0: rain
     * adds water at rest; evaporation and infiltration remove water (down
     * to a dry cell) with its velocity.  Nonzero rates switch skip_dry off. */
    double rain_rate, evap_rate, infil_rate;
} swe_params;

/* What one call of swe_step reports (all reductions in FP64). */
typedef struct {
    double t;          /* simulation time after the last step (s) */
    double dt_last;    /* tau of the last step (s) */
    double mass;       /* h^2 * sum of H after the last step (m^3) */
    double src_vol;    /* volume added by sources in the last step (m^3) */
    double clip_vol;   /* volume added by clipping negative depths, last step (m^3) */
    double max_speed;  /* max over wet cells of max(U_s, U_p) at the new state (m/s) */
    int64_t wet_cells; /* cells with H > eps_dry after the last step */
    int64_t step;      /* steps taken since swe_set_state */
    int32_t err_word;  /* device error bits (0 = none) */
    int32_t skipped;   /* work items of the last step skipped as dry (skip_dry) */
} swe_step_info;

/* Fill p with defaults: g 9.81, K 0.3, eps 1e-4, dt_max 1, FP32, fused,
 * rho_a/rho 1.225e-3, everything else 0.  nx, ny, dx must still be set. */
SWE_API void swe_params_default(swe_params* p);

/* Create a context for one grid (Sec. 2.2: uniform Cartesian grid).
 * Allocates the padded state, statics and control block on the current
 * CUDA device; bed = 0, Manning n = 0, no sources, no state yet.
 * Errors: SWE_ERR_ARG (bad sizes/parameters), SWE_ERR_OOM, SWE_ERR_CUDA. */
SWE_API int swe_create(const swe_params* p, swe_ctx** out_ctx);

/* Terrain b(x, y) and Manning roughness n_M (Sec. 2.2, Eq. 4), each nx*ny
 * host FP64.  manning_n may be NULL (0 everywhere).  Finite values only
 * (SWE_ERR_NONFINITE otherwise); |b| < 1e20. */
SWE_API int swe_set_terrain(swe_ctx* ctx, const double* b, const double* manning_n);

/* For a ghost_ring context: bed and Manning n over the whole padded extent,
 * host FP64 [ny + 2 SWE_PAD][nx + 2 SWE_PAD] row-major (the interior starts
 * at row and column SWE_PAD); manning_n may be NULL (0).  A ring cell whose
 * bed is at least 1e29 stays a wall. */
SWE_API int swe_set_terrain_ext(swe_ctx* ctx, const double* b_ext, const double* manning_n_ext);

/* State at time t: depth H >= 0 and momentum Qx = H Ux, Qy = H Uy (the
 * paper's H and HV), nx*ny host FP64 each.  Resets the step counter, the
 * time to t, and computes the first time step's signal speed (K3).
 * Errors: SWE_ERR_ARG (negative depth), SWE_ERR_NONFINITE. */
SWE_API int swe_set_state(swe_ctx* ctx, const double* H, const double* Qx, const double* Qy, double t);

/* swe_set_state with host arrays in the context's own precision (float for
 * SWE_F32, double for SWE_F64; nx*ny row-major each): copied straight into
 * the device planes by 2-D copies, half the bytes of the FP64 arrays for an
 * FP32 context and no conversion.  Same checks, errors and effects. */
SWE_API int swe_set_state_native(swe_ctx* ctx, const void* H, const void* Qx, const void* Qy, double t);

/* Sources and drains sigma with source velocity V (Eqs. 1-3).  Cell m at
 * (ix[m], iy[m]) gets sigma = weight[m] * q_{hydro[m]}(t) [m/s], evaluated
 * at t_n + tau/2, where hydrograph r has the row
 * hydro_tab[4r..4r+3] = (kind, peak, t_p, s): kind 0 is
 * peak * exp(-(t - t_p)^2 / (2 s^2)), kind 1 is the constant peak.
 * Cells must be distinct and inside the grid; vx, vy may be NULL (V = 0).
 * n = 0 removes all sources.  Copied. */
SWE_API int swe_set_sources(swe_ctx* ctx, int32_t n, const int32_t* ix, const int32_t* iy,
                    const double* weight, const double* vx, const double* vy,
                    const int32_t* hydro, int32_t n_hydro, const double* hydro_tab);

/* Open (closed[m] = 0) or close (closed[m] = 1) gate cells (hydraulic
 * structures, Sec. 1/Eq. 1 text): a closed cell is a wall, keeps its water
 * and carries no flux.  Takes effect from the next step. */
SWE_API int swe_set_solid(swe_ctx* ctx, int32_t n, const int32_t* ix, const int32_t* iy,
                  const uint8_t* closed);

/* Advance nsteps time steps (Sec. 2.3 stages I-IV, kernels K2-K8).  tau of
 * each step comes from the state at its start (K3) unless dt_fixed is set;
 * if t_end > 0 the last step is shortened to land on t_end (the reported
 * time is then t_end exactly, although in FP32 the state advanced by that
 * tau rounded to FP32) and later steps do nothing.  With info != NULL the stream is synchronised and the step
 * report copied out; device error bits turn into SWE_ERR_NONFINITE or
 * SWE_ERR_DEVICE_TIMEOUT.  With info == NULL the steps are only enqueued
 * (nsteps >= 2 run as one CUDA graph). */
SWE_API int swe_step(swe_ctx* ctx, int32_t nsteps, double t_end, swe_step_info* info);

/* Copy the current state to host FP64 arrays (any of H, Qx, Qy may be
 * NULL) and the current time to *t (may be NULL).  Synchronises. */
SWE_API int swe_get_state(swe_ctx* ctx, double* H, double* Qx, double* Qy, double* t);

/* swe_get_state into host arrays in the context's own precision (float for
 * SWE_F32, double for SWE_F64): the state's values as they are, by 2-D
 * copies.  Synchronises. */
SWE_API int swe_get_state_native(swe_ctx* ctx, void* H, void* Qx, void* Qy, double* t);

/* Device pointers of the current state (first interior cell of H, Qx, Qy),
 * the row pitch in elements and the element size in bytes.  Valid until
 * the next swe_step or swe_set_state (the state is double buffered).
 * Read only: the context keeps quantities derived from the state (the next
 * step's signal speed and, in SWE_FUSED mode, the forces of Eq. 4 per cell),
 * so a state written through these pointers would be stepped with stale
 * ones; change the state with swe_set_state. */
SWE_API int swe_get_device_ptrs(swe_ctx* ctx, void** H, void** Qx, void** Qy, int64_t* pitch_elems,
                        int32_t* elem_bytes);

/* SWE_STAGED contexts only: copy the intermediates of the last step to
 * host FP64 arrays, in the order ux, uy, ax, ay, phi, usx, usy, hs, ax2,
 * ay2, phi2, utx, uty, uhx, uhy, ht, qtx, qty, upx, upy (each nx*ny), then
 * fx [3][ny][nx+1] and fy [3][ny+1][nx] (face fluxes F_H, F_Qx, F_Qy, the
 * paper's Fh, Fv).  out[k] may be NULL to skip field k.  Synchronises. */
SWE_API int swe_get_stages(swe_ctx* ctx, double* const* out);

/* Wait for all work of the context's stream. */
SWE_API int swe_sync(swe_ctx* ctx);

/* Release every resource of the context (NULL is ignored). */
SWE_API void swe_destroy(swe_ctx* ctx);

/* Failure-path check (no counterpart in the paper): one device thread
 * waits, bounded by limit_ms (1..2000), for an mbarrier phase that nothing
 * completes -- the same bounded wait the step kernels use for their input
 * rows -- and returns SWE_ERR_DEVICE_TIMEOUT through the same error bit.
 * The device stays usable.  Any other status is a failure. */
SWE_API int swe_check_bounded_wait(int32_t limit_ms);

SWE_API const char* swe_status_str(int status);
SWE_API const char* swe_last_error(void);

/* Pick the fused kernel's rows per CTA for this grid by timing trial_steps
 * steps for each candidate (16 ... 1024 rows) on the current state, which is
 * restored afterwards (time, step counter and state unchanged).  The choice
 * does not change any result, only the speed; *seg_h_out (may be NULL)
 * receives it.  Allocates and frees a temporary copy of the state. */
SWE_API int swe_autotune(swe_ctx* ctx, int32_t trial_steps, int32_t* seg_h_out);

/* ------------------------------------------------------------------------
 * Batched ensembles.  The paper's applications need hundreds of simulations
 * of the same floodplain with different inflow hydrographs and settings of
 * tens of hydraulic structures (Sec. 1).  A batch advances n contexts
 * (scenarios of any grid sizes) together: one persistent kernel launch per
 * step hands the CTAs (scenario, tile) work items from a device list, largest
 * first; every scenario keeps its own time, time step (its own K3 max),
 * sources, walls, error word and report, and ends bitwise equal to the same
 * scenario stepped alone with swe_step (same tiling).
 * ------------------------------------------------------------------------ */
typedef struct swe_batch swe_batch; /* opaque */

/* Batch over n >= 1 distinct SWE_FUSED contexts of one precision on one
 * device, each with a state set and wall boundaries (ghost_ring = 0;
 * SWE_ERR_ARG otherwise).  The batch borrows the contexts (destroy it
 * before them) and runs on the first context's stream.  Contexts may still
 * be changed (sources, terrain, gates, state) between batch steps. */
SWE_API int swe_batch_create(swe_ctx* const* ctxs, int32_t n, swe_batch** out);

/* Gate toggles applied on the device inside the batch's step sequence:
 * event m closes (closed[m] = 1) or opens cell (ix[m], iy[m]) of scenario
 * scen[m] just before batch step step[m] (counted from the batch's creation),
 * then recomputes that scenario's time-step speed, exactly as swe_set_solid
 * between two swe_step calls would.  Replaces earlier events. */
SWE_API int swe_batch_set_gate_events(swe_batch* b, int32_t n, const int32_t* scen, const int32_t* ix,
                                      const int32_t* iy, const int64_t* step, const uint8_t* closed);

/* Advance every scenario nsteps steps (one CUDA graph: per step, the gate
 * events due, then one batched launch).  With infos != NULL (n entries) the
 * stream is synchronised and each scenario's report copied out. */
SWE_API int swe_batch_step(swe_batch* b, int32_t nsteps, swe_step_info* infos);

/* Autotuner: one rows-per-CTA value for all scenarios, chosen by timing
 * trial_steps batched steps per candidate; states are restored. */
SWE_API int swe_batch_autotune(swe_batch* b, int32_t trial_steps, int32_t* seg_h_out);

SWE_API void swe_batch_destroy(swe_batch* b);

/* ------------------------------------------------------------------------
 * Two-level nesting (the paper's hierarchical grid system with feedback,
 * Sec. 2.2, Fig. 1): a fine patch, 4x finer than its coarse parent, runs
 * four sub-steps per coarse step.  Per coarse step: (1) the coarse grid
 * steps from t to t + tau_c; (2) before each fine sub-step s = 0..3 the
 * patch's ghost ring is filled from the coarse grid at time t + s tau_c / 4
 * (the coarse cell containing each ghost cell; coarse state linear in time;
 * ghost depth = coarse free surface minus the fine bed, ghost velocity = the
 * coarse one; dry or wall coarse cells give dry ghosts) and the patch steps;
 * (3) every coarse cell under the patch takes the 4 x 4 means of the fine
 * H, Qx, Qy (feedback), and the coarse time-step speed is recomputed.  Face
 * fluxes across the patch boundary are not re-matched between the levels.
 * ------------------------------------------------------------------------ */
typedef struct swe_nest swe_nest; /* opaque */

/* Nest `fine` into `coarse` with fine interior cell (0, 0) in coarse cell
 * (ix0, iy0).  Requirements (SWE_ERR_ARG otherwise): both SWE_FUSED, one
 * precision, states set at the same time; fine->ghost_ring = 1 and coarse's
 * 0; fine nx, ny multiples of 4 and fine dx = coarse dx / 4; fixed steps with
 * fine dt_fixed = coarse dt_fixed / 4; the patch and the 3 coarse cells
 * around it inside the coarse grid.  The nest borrows both contexts (destroy
 * it before them). */
SWE_API int swe_nest_create(swe_ctx* coarse, swe_ctx* fine, int32_t ix0, int32_t iy0, swe_nest** out);

/* Advance ncoarse coarse steps (4 fine sub-steps each).  With info_coarse /
 * info_fine != NULL the streams are synchronised and the reports of both
 * grids copied out. */
SWE_API int swe_nest_step(swe_nest* n, int32_t ncoarse, swe_step_info* info_coarse, swe_step_info* info_fine);

SWE_API void swe_nest_destroy(swe_nest* n);

/* ------------------------------------------------------------------------
 * Learned closure for a 4x coarser grid level.  The paper simulates on
 * hierarchical grids, a coarse grid for deep channels and finer grids where
 * the flow needs them (Sec. 2.2, Fig. 1), with fine-to-coarse feedback; it
 * gives no closure model.  This library adds one: a 4-layer network of 3x3
 * convolutions, channels 5 -> 32 -> 32 -> 32 -> 3 with ReLU between layers,
 * that maps standardised coarse inputs (H, Ux, Uy, b, n_M) to corrections of
 * the coarse cells' net face-flux sums (the Fh, Fv of K8).  Convolutions and
 * weight gradients run on the tensor cores with BF16 weights and activations
 * and FP32 accumulation.  Their device waits are bounded: a wait that gives
 * up sets a device error word, which every later call that synchronises
 * (set/get_params, gradients, train_step with loss != NULL) reports as
 * SWE_ERR_DEVICE_TIMEOUT; the word stays set for the object's lifetime.
 *
 * A swe_cnn holds FP32 master parameters (flat: for each layer l, weights
 * [3][3][c_l][c_{l+1}] then biases [c_{l+1}]), Adam moments and the
 * activation buffers of one batch shape: n images of h x w pixels (h a
 * multiple of 8, w a multiple of 16).  Inputs x are device BF16
 * [n][h][w][16] (channels 5..15 zero); targets and outputs are device FP32
 * [n][h][w][3].  Runs on `stream` (NULL: a stream the object owns).
 * ------------------------------------------------------------------------ */
typedef struct swe_cnn swe_cnn; /* opaque */
SWE_API int swe_cnn_create(int32_t n, int32_t h, int32_t w, void* stream, swe_cnn** out);
SWE_API int swe_cnn_num_params(const swe_cnn* c);
/* Parameters from/to host FP32 (setting them resets the Adam moments). */
SWE_API int swe_cnn_set_params(swe_cnn* c, const float* params);
SWE_API int swe_cnn_get_params(swe_cnn* c, float* params);
/* Forward pass; y (device FP32 [n][h][w][3]) may be NULL. */
SWE_API int swe_cnn_forward(swe_cnn* c, const void* x, float* y);
/* Mean-squared-error loss against target and its gradient with respect to
 * every parameter (host FP32, flat layout); synchronises. */
SWE_API int swe_cnn_gradients(swe_cnn* c, const void* x, const float* target, float* grads, double* loss);
/* One training step: forward, loss, backward, Adam (beta 0.9/0.999, eps 1e-8,
 * learning rate lr).  loss may be NULL (then nothing is synchronised). */
SWE_API int swe_cnn_train_step(swe_cnn* c, const void* x, const float* target, float lr, double* loss);
SWE_API void swe_cnn_destroy(swe_cnn* c);

/* Coarse state := 4x4 block means of the fine state (H, Qx, Qy: mass and
 * momentum preserving), time := the fine time, step counter 0; fine is
 * exactly 4x coarse in both directions.  Synchronises both streams. */
SWE_API int swe_restrict_state(swe_ctx* fine, swe_ctx* coarse);
/* Standardised network inputs of the context's state into x (device BF16
 * [ny][nx][16]); norm_in = mu[5], sd[5] (host).  Synchronises. */
SWE_API int swe_closure_features(swe_ctx* ctx, const float* norm_in, void* x);
/* Standardised training targets into t (device FP32 [ny][nx][3]): the flux-
 * sum corrections (ref - pred) h / tau that turn the coarse step just taken
 * by `pred` into the restricted fine state held by `ref`; norm_out = mu[3],
 * sd[3] (host).  Synchronises. */
SWE_API int swe_closure_targets(swe_ctx* pred, swe_ctx* ref, const float* norm_out, float* t);
/* Attach (cnn != NULL) or detach a trained network of batch shape
 * (1, ny, nx) to a fused context, with norm = input mu[5], sd[5] (sd > 0),
 * output mu[3], sd[3] (sd >= 0; a channel with mu = sd = 0 adds no
 * correction) (host).  The context borrows the network. */
SWE_API int swe_closure_attach(swe_ctx* ctx, swe_cnn* cnn, const float* norm);
/* Bound the attached network's corrections (no counterpart in the paper, a
 * reading of how a learned closure may act): with beta > 0 each correction
 * c of a cell's net flux sum f (Fh, Fv_x or Fv_y of the plain step) is
 * applied as min(max(c, -beta |f|), beta |f|), so it never exceeds that
 * fraction of the flux it corrects and adds nothing where the plain step
 * moves nothing; beta = 0 (the default) applies the corrections unbounded.
 * SWE_ERR_ARG for a negative or non-finite beta.  Synchronises. */
SWE_API int swe_closure_bound(swe_ctx* ctx, double beta);
/* Closed coarse steps: per step, the network predicts corrections of the net
 * face-flux sums from the state at t_n, their depth part is centred over
 * wet cells (the corrections add no mass), and the fused step adds them in
 * its final update (K8).  nsteps >= 2 run as one CUDA graph. */
SWE_API int swe_step_closed(swe_ctx* ctx, int32_t nsteps, swe_step_info* info);

/* ------------------------------------------------------------------------
 * Allocation-free step.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory -- programs whose
 * device memory all comes from a host framework's own pool or arena, that
 * run under a fixed device-memory budget, or that must not call cudaMalloc
 * or cudaFree because those calls can synchronise the whole device.  It
 * performs one FP32 time step with the same fused kernel as swe_step and
 * calls no cudaMalloc, cudaFree or other allocating routine.
 *
 * Planes: H, Qx, Qy (state at time t), b, n (bed, Manning) and the outputs
 * H_out, Qx_out, Qy_out are caller-owned FP32 device arrays in this
 * library's padded layout: ny + 2*SWE_PAD rows of `pitch` floats, with
 * pitch >= nx + 2*SWE_PAD and a multiple of 4, each array starting on a
 * 16-byte boundary; cell (i, j) is element (j + SWE_PAD) * pitch + i +
 * SWE_PAD.  The SWE_PAD-wide ring around the grid must hold H = Qx = Qy = 0,
 * n = 0 and b >= 1e30 (walls; a closed gate is a cell with b >= 1e30).  The
 * step writes the grid's cells of the outputs only; the outputs must not
 * overlap the inputs.  No sources.
 *
 * Time step: tau = dt_fixed if p->dt_fixed > 0, else min(dt_max, cfl * dx /
 * max_speed) with max_speed the largest signal speed of the input state,
 * i.e. the max_speed reported for it by swe_step or by the previous call of
 * this function (0 for still water); max_speed < 0 without dt_fixed is
 * rejected.  With info != NULL the stream is synchronised and the report
 * (new t, tau, mass, wet cells, max_speed of the output state) filled, and
 * device-side failures are returned as error codes.  With info == NULL the
 * call only enqueues the step and reports nothing: a device error (a
 * bounded wait that ran out, a non-finite signal speed, a non-positive
 * step), the new t and the max_speed the next call needs are then lost,
 * since the next call clears the control block they live in.  So pass info
 * unless dt_fixed > 0 and the caller checks the output state another way.
 * Runs on p->cuda_stream (NULL: the legacy default stream).
 *
 * Scratch: the kernel's control block, one partial-sum record per CTA and
 * an empty source table live in a file-scope device array of
 * SWE_NOALLOC_SCRATCH_BYTES bytes that every GPU loading this library keeps
 * until the process exits.  Grids needing more than SWE_NOALLOC_MAX_ITEMS
 * CTAs (nx > 7000 * 116 cells) are rejected with SWE_ERR_ARG.  The first
 * call on a device looks up the array's device address and sets the
 * kernel's shared-memory size (once per device); make that first call
 * before any stream capture.  Every call resets what must start at zero,
 * but all calls share the one array: calls whose work can overlap on the
 * GPU (other streams, other host threads) race and corrupt each other's
 * results, so serialise them.
 * Errors: SWE_ERR_ARG (sizes, alignment, layout, a pitch above INT_MAX,
 * parameters; checked before any device work), SWE_ERR_CUDA, and, with
 * info != NULL only, SWE_ERR_NONFINITE, SWE_ERR_DT, SWE_ERR_DEVICE_TIMEOUT.
 * ------------------------------------------------------------------------ */
#define SWE_PAD 10
#define SWE_NOALLOC_MAX_ITEMS 7000
#define SWE_NOALLOC_SCRATCH_BYTES 252416
SWE_API int swe_step_f32_noalloc(const swe_params* p, const float* H, const float* Qx, const float* Qy,
                                 const float* b, const float* n, float* H_out, float* Qx_out,
                                 float* Qy_out, int64_t pitch, double t, double max_speed,
                                 swe_step_info* info);

#ifdef __cplusplus
}
#endif

#endif /* SWE_H */
