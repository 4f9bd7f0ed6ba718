/*
 * cx.h -- C ABI of the GB300 time-stepper for the bacteria/nutrient
 * chemotaxis system with degenerate cross diffusion (Leyva, Malaga & Plaza).
 *
 * The library integrates, on one GPU, the dimensionless system of
 * Sec. 2.4 (Eq. ka-chem-model), written in its general form with the
 * nutrient diffusivity Dn and conversion factor theta of Eq. ka-model-dim:
 *
 *   n_t = Dn Lap(n) - n b                                        (Eq. eqnadim)
 *   b_t = div(sigma n b grad b) + theta n b
 *         - div(chi(n) sigma n b^2 grad n)                       (Eq. eqbadim)
 *   chi(n) = chi0 / (1 + n)^2   (receptor law, Eq. receptor_law)
 *         or chi0               (constant law, Eq. velo-system)
 *   sigma  = sigma0 (1 + a Delta)                                (Eq. CoefCrsDif)
 *
 * on an nx*ny cell-centred grid of spacing dx with no-flux walls
 * (Eq. bconds), initial data n = n0 and b = bM exp(-r^2/r0sq), cut to zero
 * where r^2/r0sq > 40 (Eq. inicond, Eq. inibacexp), by explicit finite volumes (face fluxes with arithmetic
 * face means) and forward Euler or Heun time stepping (Sec. 3).
 *
 * Conventions for every call:
 *   - return CX_OK (0) on success, a negative CX_ERR_* code on failure; no
 *     call throws and no call aborts the process;
 *   - cx_last_error() returns a message for the last failure on the
 *     calling thread;
 *   - handles own every device buffer they allocate; the caller owns every
 *     host pointer it passes and may reuse it when the call returns;
 *   - host arrays are row-major: element (i, j) is at [j*nx + i], i along x;
 *   - NULL handles are rejected with CX_ERR_INVALID_ARG (cx_destroy and
 *     cx_batch_destroy accept NULL and do nothing).
 */
#ifndef CX_H
#define CX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CX_VERSION 1

/* status codes */
#define CX_OK 0
#define CX_ERR_INVALID_ARG (-1)  /* bad pointer, size, enum or parameter value */
#define CX_ERR_DT_UNSTABLE (-2)  /* dt above the explicit stability limit */
#define CX_ERR_OOM (-3)          /* device or pinned-host allocation failed */
#define CX_ERR_CUDA (-4)         /* a CUDA runtime call failed */
#define CX_ERR_NONFINITE (-5)    /* diagnostics found a NaN or Inf */
#define CX_ERR_NEGATIVE (-6)     /* diagnostics found b < 0 or n < 0 */
#define CX_ERR_TIMEOUT (-7)      /* a bounded device-side wait ran out */
#define CX_ERR_IO (-8)           /* checkpoint file could not be read/written */
#define CX_ERR_UNSUPPORTED (-9)  /* option combination not built */

/* field selectors */
#define CX_FIELD_B 0
#define CX_FIELD_N 1
#define CX_FIELD_SIGMA 2

/* host element types for field I/O */
#define CX_F64 0
#define CX_F32 1

/* option values */
#define CX_CHEMO_RECEPTOR 0   /* chi0 / (1+n)^2 at the face */
#define CX_CHEMO_CONSTANT 1   /* chi0 */
#define CX_MOBILITY_CENTRAL 0 /* b^2 at a face = ((b_L+b_R)/2)^2 */
#define CX_MOBILITY_UPWIND 1  /* b^2 at a face = b^2 of the lower-n cell */
#define CX_NOISE_UNIFORM 0    /* Delta uniform on [-1,1) */
#define CX_NOISE_TRIANGULAR 1 /* Delta triangular on (-1,1) (Sec. 3) */
#define CX_NOISE_STATIC 0     /* sigma drawn once, at time step 0 */
#define CX_NOISE_PER_STEP 1   /* sigma redrawn for every time step (Sec. 3) */
#define CX_SCHEME_EULER 0     /* u' = u + dt r(u) */
#define CX_SCHEME_HEUN 1      /* u' = u + dt/2 (r(u) + r(u + dt r(u))) */
#define CX_PREC_F64 0         /* state and arithmetic in FP64 */
#define CX_PREC_F32 1         /* state and arithmetic in FP32; diagnostics in FP64 */

typedef struct cx_ctx cx_ctx;     /* one simulation; owns its device buffers */
typedef struct cx_batch cx_batch; /* many independent simulations */

/* Grid: nx*ny cells of side dx.  Cell (i,j) has its centre at
 * x = (i + 1/2 - nx/2) dx, y = (j + 1/2 - ny/2) dx (inoculum at the origin). */
typedef struct {
    int32_t nx, ny;
    double dx;
} cx_grid;

/* Model and numerical parameters (Sec. 2.4 free parameters sigma0, n0,
 * chi0; Dn and theta of Eq. ka-model-dim, 1 in the normalised form). */
typedef struct {
    double n0;          /* initial nutrient level (Eq. inicond) */
    double chi0;        /* chemotactic strength, >= 0 */
    double sigma0;      /* mean motility (agar softness), >= 0 */
    double noise_amp;   /* a in sigma = sigma0 (1 + a Delta), 0 <= a <= 1 */
    double Dn;          /* nutrient diffusivity, >= 0 */
    double theta;       /* conversion factor, >= 0 */
    double bM;          /* inoculum peak (Eq. inibacexp) */
    double r0sq;        /* inoculum width: b = bM exp(-r^2 / r0sq) where
                           r^2 / r0sq <= 40, else 0 (compact support), > 0 */
    double dt;          /* time step; 0 selects cfl_frac * cx_dt_limit() */
    double cfl_frac;    /* fraction of the limit used when dt == 0, (0, 1] */
    double b_threshold; /* envelope level for r_env; <= 0 selects 0.1 theta n0 */
    int32_t chemo_law;  /* CX_CHEMO_* */
    int32_t mobility;   /* CX_MOBILITY_* */
    int32_t noise_dist; /* CX_NOISE_UNIFORM / CX_NOISE_TRIANGULAR */
    int32_t noise_mode; /* CX_NOISE_STATIC / CX_NOISE_PER_STEP */
    int32_t scheme;     /* CX_SCHEME_* */
    int32_t precision;  /* CX_PREC_* */
} cx_params;

/* Diagnostics of the current state (every sum accumulated in FP64). */
typedef struct {
    int64_t step;     /* time steps taken */
    double t;         /* step * dt */
    double dt;
    double mass_b;    /* dx^2 sum b */
    double mass_n;    /* dx^2 sum n */
    double invariant; /* dx^2 sum (b + theta n): conserved (Eq. mass-conser) */
    double min_b, min_n, max_b;
    double r_env;     /* largest cell-centre distance with b >= b_threshold, 0 if none */
    int32_t finite;   /* 1 if every b and n is finite */
    int32_t status;   /* CX_OK, CX_ERR_NONFINITE or CX_ERR_NEGATIVE */
    double area_env;  /* dx^2 x the number of cells with b >= b_threshold: the area
                         of the colony, whose equivalent radius sqrt(area_env / pi)
                         averages the front over every direction */
} cx_diag;

/* ---- host-only helpers (no GPU needed) ---------------------------------- */

/* Library version (CX_VERSION of the build). */
int cx_version(void);

/* Static text for a status code; never NULL. */
const char *cx_strerror(int code);

/* Message of the last failure on this thread ("" if none); valid until the
 * next failing call on the same thread. */
const char *cx_last_error(void);

/* Fill *p with the normalised model (Dn = theta = 1), receptor law, central
 * mobility, static uniform noise a = 0.5, Euler, FP32, dt = 0.2 x limit,
 * n0 = 0.71, sigma0 = 1, chi0 = 0, bM = 0.71, r0sq = 6.25 (Sec. 3). */
int cx_params_default(cx_params *p);

/* Explicit stability limit for (g, p) (Sec. 3 only states that its steps
 * were stable; this library's reading):
 *   B = bM + theta n0,  Dmax = max(Dn, sigma0 (1+a) n0 B (1 + chi0 B)),
 *   limit = min(dx^2 / (4 Dmax), 1 / (4 Dn / dx^2 + B)).
 * Validates g and p; writes *limit. */
int cx_dt_limit(const cx_grid *g, const cx_params *p, double *limit);

/* ---- one simulation ------------------------------------------------------ */

/* Allocate a simulation on the current CUDA device, draw sigma from
 * Philox4x32-10 keyed by `seed` (cell index and time step as counter;
 * Salmon et al., SC'11) and set the initial state.  Synchronous.
 * Errors: INVALID_ARG (bad grid/params/out), DT_UNSTABLE (p->dt above the
 * limit), OOM, CUDA.  On error *out is left NULL. */
int cx_create(const cx_grid *g, const cx_params *p, uint64_t seed, cx_ctx **out);

/* As cx_create, over device arrays the caller owns (e.g. tensors of a
 * framework whose allocator owns the device memory): b[0], b[1] and n[0],
 * n[1] (the ping-pong state) and sigma, each ny rows of `pitch` elements of
 * the state precision (FP32 or FP64 per p->precision) on the current device.
 * The handle initialises them as cx_create does (sigma field, inoculum; the
 * second state buffers zeroed) and never frees them: they must outlive the
 * handle.  Which of b[0] / b[1] holds the current state changes with every
 * pass, and inside each row the library keeps every aligned group of four
 * cells in the order (4g, 4g+2, 4g+1, 4g+3) (the pair order, which lets a
 * 16-byte load feed the paired arithmetic directly): read and write the
 * fields through cx_get_field / cx_set_field, which give the natural order.
 * Requirements: every pointer non-NULL and 16-byte aligned, pitch >= nx and
 * a multiple of 4 elements (a multiple of 128 bytes is fastest), and no two
 * arrays overlapping.  Errors: INVALID_ARG (checked before any device work),
 * DT_UNSTABLE, CUDA.  There is no counterpart in the paper (a memory-ownership
 * interface). */
int cx_create_with_buffers(const cx_grid *g, const cx_params *p, uint64_t seed, void *const b[2],
                           void *const n[2], void *sigma, int64_t pitch, cx_ctx **out);

/* Run all later work of `c` on `stream` (a cudaStream_t, e.g. a torch
 * stream handle; NULL = the legacy default stream). */
int cx_set_stream(cx_ctx *c, void *stream);

/* Advance by n_steps >= 0 time steps.  Asynchronous on the handle's stream:
 * kernel launches only, no host synchronisation.  Errors: INVALID_ARG, CUDA
 * (launch failures). */
int cx_step(cx_ctx *c, int64_t n_steps);

/* Wait for all queued work of the handle. */
int cx_synchronize(cx_ctx *c);

/* Reduce the current state (FP64 sums, deterministic order) and copy the
 * result to *out.  Synchronises the handle's stream.  Returns CX_OK, or
 * CX_ERR_NONFINITE / CX_ERR_NEGATIVE with *out filled when the state is
 * unhealthy, or INVALID_ARG / CUDA. */
int cx_diagnostics(cx_ctx *c, cx_diag *out);

/* Copy field `which` (CX_FIELD_*) to the host array `host` of `count`
 * elements (count must equal nx*ny) of type `dtype` (CX_F64/CX_F32),
 * converting if the state precision differs.  Synchronous. */
int cx_get_field(cx_ctx *c, int32_t which, void *host, int32_t dtype, size_t count);

/* Overwrite field `which` from a host array (same layout rules as
 * cx_get_field).  Synchronous with respect to `host`.  Replacing sigma is
 * allowed only with CX_NOISE_STATIC (per-step noise regenerates it). */
int cx_set_field(cx_ctx *c, int32_t which, const void *host, int32_t dtype, size_t count);

/* Staged upload of a new state (b and n), overlapping the copies with the
 * handle's queued work.  cx_stage_state starts host-to-device copies of the
 * nx*ny arrays `b_host` and `n_host` (row-major, dtype = the state's own
 * type, CX_F32 or CX_F64; no conversion) into staging arrays the handle
 * owns, on a copy stream of its own, and returns without waiting: the copies
 * are asynchronous when the host arrays are pinned (e.g. cudaMallocHost or a
 * pinned torch tensor), and the caller must keep the arrays valid and
 * unchanged until the next cx_commit_state has been followed by a
 * synchronising call (cx_diagnostics, cx_synchronize, ...).  The first call
 * allocates the staging arrays (two more state-sized arrays).
 * cx_commit_state makes the staged arrays the current b and n for all work
 * queued after it: the handle's stream waits for the staged copies (no host
 * wait), then the arrays swap roles (a device-to-device copy instead when the
 * state arrays are the caller's, cx_create_with_buffers).  The step counter
 * and time are unchanged, as with cx_set_field.  A later cx_stage_state
 * waits, on the copy stream, until the work queued before the last commit is
 * done with the arrays it overwrites.  Errors: INVALID_ARG (NULL pointers,
 * wrong dtype or count, a second stage before the commit, a commit with
 * nothing staged), OOM/CUDA. */
int cx_stage_state(cx_ctx *c, const void *b_host, const void *n_host, int32_t dtype, size_t count);
int cx_commit_state(cx_ctx *c);

/* Copy the handle's grid, parameters (with dt resolved) and seed; any
 * output pointer may be NULL. */
int cx_get_config(cx_ctx *c, cx_grid *g, cx_params *p, uint64_t *seed);

/* Current step count, time and time step. */
int cx_get_time(cx_ctx *c, int64_t *step, double *t, double *dt);

/* Reset the step counter (the time is step * dt); used with cx_set_field to
 * restart from given data. */
int cx_set_step(cx_ctx *c, int64_t step);

/* Height in rows of one step-kernel tile (each CTA marches one tile of
 * 512 columns x rows; with two stages per pass, 120 x rows per one-warp
 * CTA, or 480 x rows per four-warp CTA when sigma is redrawn every step), 1..4096 with
 * ceil(ny/rows) <= 65535, or 0 for the automatic height; a performance
 * knob that the autotuner sets.  The result is bit-identical for every
 * value.  Automatic: 32 rows (64 with two stages per pass), or fewer on
 * small grids so that about four tiles per SM are launched (sixteen
 * one-warp tiles with two stages and static sigma, eight four-warp tiles
 * with sigma redrawn per step); cx_get_tile_rows reports the height in
 * effect. */
int cx_set_tile_rows(cx_ctx *c, int32_t rows);
int cx_get_tile_rows(cx_ctx *c, int32_t *rows);

/* Temporal blocking depth: the number of explicit stages of Eq. ka-chem-model
 * that one pass over the grid takes, 1 or 2.  At 2, cx_step runs two
 * forward-Euler steps per pass (an odd remainder takes a single pass), or
 * both stages of a Heun step in one pass, the intermediate state held in
 * registers; a pass then reads and writes the state once for two stages.
 * The result is bit-identical for both values (the stages evaluate the same
 * operations on the same operands) and the stability limit is that of one
 * step.  A performance knob; default 2 for an FP32 state, 1 for FP64 (whose
 * pass is bound by the FP64 pipe).  Errors: INVALID_ARG. */
int cx_set_time_block(cx_ctx *c, int32_t stages);
int cx_get_time_block(cx_ctx *c, int32_t *stages);

/* Write / read a checkpoint: header (grid, params, seed, step, dt,
 * precision) and the raw b, n and sigma arrays.  A run resumed from a
 * checkpoint continues bit for bit as the uninterrupted run.  Errors: IO,
 * INVALID_ARG, OOM, CUDA. */
int cx_save(cx_ctx *c, const char *path);
int cx_load(const char *path, cx_ctx **out);

/* Free the handle and its device buffers.  NULL is a no-op. */
void cx_destroy(cx_ctx *c);

/* ---- many simulations at once (parameter sweeps) --------------------------
 *
 * A batch holds `count` independent simulations of the same system with
 * their own grid size, parameters (n0, chi0, sigma0, a, ...) and seed, as in
 * the parameter study of Sec. 3 (Table tabresparam).  All instances share
 * precision, scheme, chemo_law, mobility and noise_mode.  With
 * CX_NOISE_PER_STEP (the paper's own runs, Sec. 3: sigma redrawn at every
 * point and time step) each instance draws sigma from (its seed, cell, time
 * step) as a single grid does; the batch keeps the time step in a device
 * word that it writes before each captured graph or run of passes, so the
 * graphs stay valid across calls.  An instance evolves bit for bit as a
 * cx_ctx created with the same grid, parameters and seed.  A batch owns a
 * non-default CUDA stream. */

/* Allocate and initialise `count` instances (1..65535); grids[i],
 * params[i], seeds[i] describe instance i.  Synchronous.  Errors:
 * INVALID_ARG (including instances that differ in precision, scheme,
 * chemo_law, mobility or noise_mode), DT_UNSTABLE, OOM, CUDA. */
int cx_batch_create(int32_t count, const cx_grid *grids, const cx_params *params,
                    const uint64_t *seeds, cx_batch **out);

/* Run later work on `stream` (a non-default cudaStream_t). */
int cx_batch_set_stream(cx_batch *b, void *stream);

/* Performance knobs, none of which changes any result bit:
 *   tile_rows   rows per tile of the step kernel (1..4096; the tiles of
 *               both depths; default 128 for FP32 batches, which take two
 *               stages per pass, 32 for FP64 ones);
 *   graph_steps steps captured per CUDA graph and replayed (0: plain
 *               launches; rounded up to even for Euler; default 64);
 *   group_bytes if > 0, instances are cut into consecutive groups whose
 *               fields fit this many bytes and each group runs all its steps
 *               before the next starts (keeps a group resident in L2);
 *               0: every launch covers every instance (default);
 *   resident_steps if > 0, each group advances up to this many steps per
 *               launch: one cooperative launch whose resident blocks share
 *               the group's tiles and meet at a grid barrier between steps
 *               (the fields stay in L2 across steps); 0: one launch per step
 *               (default).  Every barrier wait is bounded: if one runs out
 *               (a fault, never in normal operation), the next
 *               cx_batch_synchronize / cx_batch_diagnostics returns
 *               CX_ERR_TIMEOUT and the batch state is undefined. */
int cx_batch_set_tuning(cx_batch *b, int32_t tile_rows, int32_t graph_steps, int64_t group_bytes,
                        int32_t resident_steps);
int cx_batch_get_tuning(cx_batch *b, int32_t *tile_rows, int32_t *graph_steps, int64_t *group_bytes,
                        int32_t *resident_steps);

/* Temporal blocking depth of the batch, as cx_set_time_block: 2 takes two
 * Euler steps (or one whole Heun step) per pass over every instance, on
 * 120-column one-warp tiles; 1 one step per pass.  Results are bit-identical for
 * both.  Default: 2 for FP32 batches, 1 for FP64.  The resident mode
 * (resident_steps > 0) takes one stage per pass whatever the depth.
 * Errors: INVALID_ARG. */
int cx_batch_set_time_block(cx_batch *b, int32_t stages);
int cx_batch_get_time_block(cx_batch *b, int32_t *stages);

/* Advance every instance by n_steps >= 0 steps.  Asynchronous. */
int cx_batch_step(cx_batch *b, int64_t n_steps);
int cx_batch_synchronize(cx_batch *b);

/* Diagnostics of every instance into out[0..count-1] (FP64 sums; the
 * summation order differs from cx_diagnostics, so sums agree to round-off).
 * Synchronises.  Returns NONFINITE / NEGATIVE (out filled, per-instance
 * status set) if an instance is unhealthy. */
int cx_batch_diagnostics(cx_batch *b, cx_diag *out);

/* Field I/O of instance `index` (same rules as cx_get_field/cx_set_field). */
int cx_batch_get_field(cx_batch *b, int32_t index, int32_t which, void *host, int32_t dtype,
                       size_t count);
int cx_batch_set_field(cx_batch *b, int32_t index, int32_t which, const void *host,
                       int32_t dtype, size_t count);

/* Number of instances and steps taken. */
int cx_batch_get_time(cx_batch *b, int32_t *count, int64_t *step);

/* Free the batch.  NULL is a no-op. */
void cx_batch_destroy(cx_batch *b);

/* ---- morphology labels ----------------------------------------------------
 *
 * b sampled at nsamples points of the circle of `radius` (physical units)
 * about the domain centre, sample k at angle 2 pi k / nsamples, by bilinear
 * interpolation of the cell-centred values (clamped at the walls), into
 * host_out[0..nsamples).  The number of circular runs above the envelope
 * level at radius 0.8 r_env is the colony's branch count (the paper reads
 * branch numbers off its figures, Sec. 3).  Synchronous. */
int cx_polar_profile(cx_ctx *c, double radius, int32_t nsamples, double *host_out);
int cx_batch_polar_profile(cx_batch *b, int32_t index, double radius, int32_t nsamples,
                           double *host_out);

/* ---- surrogate network ----------------------------------------------------
 *
 * An ensemble of E independent MLPs 4 -> 256 -> 256 -> 2 with tanh hidden
 * units that map a sweep point (normalised n0, chi0, sigma0, a) to
 * normalised morphology labels (envelope velocity, branch count), trained
 * on data the solver produces.  The 256 x 256 layer and its two backward
 * products run on the tensor cores (tcgen05, bf16 operands, FP32
 * accumulation in tensor memory); everything else is FP32.  One member's
 * parameters are FP32, packed as W1 (256 x 4, row-major), b1 (256), W2
 * (256 x 256), b2 (256), W3 (2 x 256), b3 (2): CX_MLP_PARAMS floats; the
 * members' blocks follow one another (member-major).  Loss = sum (Y - T)^2
 * / (2 B).  Member e of an E-member network computes, bit for bit, what a
 * one-member network with member e's parameters and data computes.  The
 * paper has no counterpart: the network only proposes and pre-screens sweep
 * points; every reported label comes from the solver.
 *
 * Every call below is synchronous and returns CX_ERR_TIMEOUT if a bounded
 * device-side wait for the tensor cores ran out (the results of that call
 * are then undefined; the network stays usable).  The environment variable
 * CX_MMA_WAIT_LIMIT, read when a network is created, sets the number of
 * polls of that wait (default 2^22). */
#define CX_MLP_PARAMS 67586
typedef struct cx_mlp cx_mlp;

/* Allocate a network of `members` (1..64) members for batches of up to
 * max_batch rows (1..2^20); the parameters start at zero (set them with
 * cx_mlp_set_params).  Device memory: about members x max_batch x 5.7 KB
 * (the activations of the backward pass). */
int cx_mlp_create_members(int32_t max_batch, int32_t members, cx_mlp **out);
/* cx_mlp_create_members(max_batch, 1, out). */
int cx_mlp_create(int32_t max_batch, cx_mlp **out);
/* Number of members (0 for NULL). */
int32_t cx_mlp_members(const cx_mlp *m);
/* Set / read all parameters (count == members x CX_MLP_PARAMS); setting
 * them also resets the optimiser state. */
int cx_mlp_set_params(cx_mlp *m, const float *host, size_t count);
int cx_mlp_get_params(cx_mlp *m, float *host, size_t count);
/* Every member on the same inputs: x (batch x 4) -> y (members x batch x 2),
 * host arrays. */
int cx_mlp_forward(cx_mlp *m, const float *x, int32_t batch, float *y);
/* Loss and gradient of every member on the same batch (x, t): grad receives
 * members x CX_MLP_PARAMS floats (same packing), loss (optional) members
 * doubles. */
int cx_mlp_gradient(cx_mlp *m, const float *x, const float *t, int32_t batch, float *grad,
                    double *loss);
/* `steps` Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, rate lr) of every
 * member over minibatches of `batch` consecutive rows of its own n-row set,
 * taken cyclically (shuffle the rows beforehand): x is members x n x 4, t
 * members x n x 2 (member-major).  loss_out (optional, members x steps
 * doubles) receives each member's minibatch losses. */
int cx_mlp_train(cx_mlp *m, const float *x, const float *t, int32_t n, int32_t batch,
                 int32_t steps, float lr, double *loss_out);
/* Free the network.  NULL is a no-op. */
void cx_mlp_destroy(cx_mlp *m);

/* ---- diagnostics without any allocation --------------------------------- */

/* The paper has no counterpart to this call; it exists for callers that may
 * not allocate device or pinned memory themselves.  Examples: a framework
 * whose caching allocator owns all device memory (a stray cudaMalloc or
 * cudaFree synchronises the whole device and fragments that pool), a
 * service that sized its device memory once at start-up and must stay
 * within that budget, or a time-critical loop in which a blocking
 * allocation is not allowed.
 *
 * It computes the same reduction as cx_diagnostics, with the same kernels,
 * over fields the caller owns, in natural in-row order (the library's own
 * arrays keep each group of four cells in pair order, so the summation order
 * within a row differs and the sums agree to round-off):
 *   b, n        device arrays of nx*ny cells, row j at element j*pitch,
 *               FP64 or FP32 as `precision` (CX_PREC_*) says;
 *   pitch       elements per row, >= nx;
 *   dx, theta   cell size (> 0) and conversion factor (>= 0) for the
 *               masses and the invariant dx^2 sum (b + theta n);
 *   b_threshold envelope level for r_env (> 0);
 *   stream      cudaStream_t to run on (NULL = legacy default stream);
 *   result_dev  caller-owned device array of 8 doubles that receives
 *               {sum b, sum n, min b, min n, max b, max (2i+1-nx)^2 +
 *               (2j+1-ny)^2 over b >= b_threshold (-1 if none),
 *               non-finite flag, number of cells with b >= b_threshold};
 *   out         optional host struct: if non-NULL the call copies the
 *               record back, waits for `stream` and fills *out (step, t and
 *               dt are 0: there is no handle).  If NULL the call only
 *               queues work on `stream` and returns.
 * The per-block partial records live in one static device array of 1024
 * records x 8 doubles (64 KiB).  The CUDA driver sets the array up when it
 * loads the library's device code on a device: at the first call on that
 * device under lazy module loading (CUDA's default), or when the library is
 * loaded if CUDA_MODULE_LOADING=EAGER; from then on the device holds it
 * until the process exits (or its context is destroyed).  That first call
 * per device may therefore make the driver allocate the module's memory;
 * every later call allocates nothing and frees nothing.  The reduction uses
 * at most 1024 blocks for any grid, so every grid within these limits fits:
 * nx, ny >= 1, nx*ny <= 2^32, nx <= 2^26 (so that record slot 5 holds the
 * squared radius exactly, below 2^53) and ny <= 2,097,120; larger sizes are
 * rejected with CX_ERR_INVALID_ARG.
 *
 * All calls share that one array and it keeps the last call's contents;
 * every record a call reads is written earlier in the same call, so nothing
 * needs clearing.  Calls that overlap on the GPU (on different streams, or
 * from different threads) race on the array and must be serialised by the
 * caller.  The first call in each device's context looks up the array's
 * device address (with that device current); make that first call before
 * any stream capture.  After cudaDeviceReset (or any destruction of the
 * device's primary context) the next call looks the address up again in
 * the new context, so it counts as a first call once more.  Errors:
 * INVALID_ARG, CUDA, and NONFINITE / NEGATIVE (with *out filled) as for
 * cx_diagnostics when `out` is given. */
int cx_diagnostics_noalloc(const void *b, const void *n, int32_t nx, int32_t ny, int64_t pitch,
                           int32_t precision, double dx, double theta, double b_threshold,
                           void *stream, double *result_dev, cx_diag *out);

/* ---- arithmetic peak of the device --------------------------------------- */

/* The paper has no counterpart to this call: it measures the denominator of
 * the step kernels' arithmetic roofline.  GB300 runs FP64 at a small
 * fraction of its FP32 rate, so an FP64 state is bound by the FP64 pipe and
 * its roofline needs that pipe's measured rate.  The call launches, on a
 * private stream of the current device, a register-only kernel in which
 * every thread advances 8 independent multiply-add chains (4 blocks of 256
 * threads per SM), once to warm up and then `repeats` times (1..100), timed
 * with CUDA events, and writes the best rate to *flops_per_s (a
 * multiply-add counts two flops).  precision: CX_PREC_F64 or CX_PREC_F32.
 * It allocates and frees one small device buffer and synchronises its
 * stream.  Errors: INVALID_ARG, CUDA. */
int cx_alu_peak(int32_t precision, int32_t repeats, double *flops_per_s);

#ifdef __cplusplus
}
#endif

#endif /* CX_H */
