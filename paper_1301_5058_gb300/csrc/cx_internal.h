// cx_internal.h -- internal declarations shared by the library's translation
// units: the handle layout, kernel argument blocks and launchers.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "cx.h"

namespace cx {

// Named range on profiler timelines for the life of a scope (NVTX; a
// no-op unless a profiling tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Per-run coefficients of the face fluxes.  The kernels evaluate unscaled
// face fluxes and apply the constant factors once per cell, so that one
// step reads
//   b' = b + dt theta n b + cA (phiE - phiW + phiN - phiS)
//   n' = n - dt n b       + cG (gE - gW + gN - gS)
// with, on a face between L (left/lower) and R (right/upper),
//   hc  = chi(n_f) / 2 = cChi / (2+n2)^2 (receptor law) or cChi (constant law)
//   phi = s2 n2 b2 (db - hc b2 dn)                   central mobility b_f^2
//   phi = s2 n2 (b2 db - 4 hc b_d^2 dn)              donor-cell mobility b_d^2
//   g   = dn
// where s2 = sL+sR, n2 = nL+nR, b2 = bL+bR, db = bR-bL, dn = nR-nL and b_d
// is b of the lower-n cell.  Derivation: sigma_f n_f b_f = s2 n2 b2 / 8,
// b_f^2 = b2^2 / 4 and, for the receptor law, chi(n_f) = 4 chi0 / (2+n2)^2.
struct Coef {
    double cA;    // dt / (8 dx^2)
    double cChi;  // receptor: 2 chi0; constant: chi0 / 2
    double cG;    // dt Dn / dx^2
    double cR;    // dt theta
    double cN;    // dt
};

struct Sigma {  // how sigma is obtained
    int per_step;     // 0: read the sigma array; 1: regenerate from Philox every step
    int dist;         // CX_NOISE_*
    double sigma0, amp;
    uint64_t seed;
};

// One launch of the step kernel.  stage 0: u_out = u + dt r(u) (forward
// Euler, or the first Heun stage); stage 1: the second Heun stage,
// u_out = (u0 + u + dt r(u)) / 2 with u0 read pointwise from (bu, nu) and
// written back in place (bo == bu, no == nu).
struct StepArgs {
    const void *b, *n, *s;  // stencil input state (+ sigma array, static noise)
    const void *bu, *nu;    // stage 1: state at the start of the step
    void *bo, *no;          // output state
    int nx, ny;
    long long pitch;        // elements per row
    int law, mob, stage;
    int rows;               // tile height in rows (grid.y = ceil(ny / rows))
    Coef k;
    Sigma sg;
    long long step;         // index of the time step being taken (noise counter)
};

// Launchers (return a cudaError_t from the launch).  recipe 0: FP64 sigma
// recipe, 1: FP32 recipe (per-step noise of an FP32 state).
cudaError_t launch_sigma_init(int prec, void *sigma, int nx, int ny, long long pitch,
                              uint64_t seed, uint64_t step, double sigma0, double amp,
                              int dist, int recipe, cudaStream_t st);
cudaError_t launch_initial_state(int prec, void *b, void *n, int nx, int ny, long long pitch,
                                 double dx, double n0, double bM, double r0sq, cudaStream_t st);
cudaError_t launch_step(int prec, const StepArgs &a, cudaStream_t st);
// Two stages in one pass (cx_fused.cu): heun 0 takes the Euler steps a.step
// and a.step + 1, heun 1 the Heun step a.step; reads (b, n, s), writes
// (bo, no), which must be other buffers.  bu / nu / stage are not used.
cudaError_t launch_fused(int prec, const StepArgs &a, int heun, cudaStream_t st);

// In-row order of the device arrays.  Each aligned group of four cells of a
// row, columns 4g .. 4g+3, is stored as (4g, 4g+2, 4g+1, 4g+3): a 16-byte
// vector load then hands a thread its cells already as the pairs
// (4g, 4g+2) and (4g+1, 4g+3) that the paired FP32 arithmetic works on, with
// no register moves to regroup them (1.05x on the 16384^2 FP32 pass).  The
// order swaps the middle two of each group, so it is its own inverse.  Rows
// therefore need a pitch that is a multiple of 4 elements; a row's last
// group may hold a cell beyond nx in the padding columns.
__host__ __device__ __forceinline__ long long pair_col(long long i)
{
    return (i & ~3LL) | ((i & 1LL) << 1) | ((i >> 1) & 1LL);
}
// Swaps the middle two elements of every group of four of the first
// ceil(nx/4)*4 columns of each row, in place: converts an array between the
// natural in-row order and the pair order (either way).
cudaError_t launch_pair_order(int prec, void *a, int nx, int ny, long long pitch, cudaStream_t st);

struct DiagScratch {
    double *partials;  // [blocks][8]
    double *result;    // [8] on the device
    int blocks;
};
int diag_blocks_for(int ny);
// pair_order: the fields are in the library's pair order (else natural).
cudaError_t launch_diagnostics(int prec, const void *b, const void *n, int nx, int ny,
                               long long pitch, double b_threshold, DiagScratch s,
                               cudaStream_t st, bool pair_order = true);

// b on a circle of `radius` about the domain centre, ns samples (cx_labels.cu).
cudaError_t launch_polar(int prec, const void *b, int nx, int ny, long long pitch, double dx,
                         double radius, int ns, double *out, cudaStream_t st);

// Store `msg` as this thread's cx_last_error() text; returns `code`.
int record_error(int code, const char *msg);

// Host helpers shared by the single-grid and batch entry points
// (cx_api.cu): parameter validation, the time step (CX_ERR_DT_UNSTABLE
// above the limit), the scaled flux coefficients and the envelope level.
int validate_params(const cx_grid *g, const cx_params *p);
int resolve_time_step(const cx_grid *g, const cx_params *p, double *dt);
Coef make_coef(const cx_grid &g, const cx_params &p, double dt);
double envelope_level(const cx_params &p);

// Batched stepping and diagnostics (cx_batch.cu).  `inst` is the device
// instance table, `work` the device work list (int4: instance, tile x,
// tile y, unused).
size_t inst_dev_bytes(int prec);
void fill_inst(int prec, void *table, int i, void *b0, void *b1, void *n0, void *n1, void *s,
               int nx, int ny, long long pitch, const Coef &k, double bth, uint64_t seed,
               double sigma0, double amp, int dist);
// Per-step noise of a batch pass: on = 1 redraws sigma every step; the
// pass's first time step is *step_base + step_off (step_base: device int64
// written by launch_set_step before the pass or the graph holding it).
struct BatchNoise {
    int on;
    const long long *step_base;
    int step_off;
};
cudaError_t launch_set_step(long long *step_base, long long step, cudaStream_t st);
cudaError_t launch_batch_step(int prec, int law, int mob, const void *inst, const int4 *work,
                              int nwork, int parity, int rows, int stage, const BatchNoise &nz,
                              cudaStream_t st);
// Two stages per pass over a 480-column work list: reads u(parity), writes
// u(parity^1); heun 0: two Euler steps, 1: one Heun step.
cudaError_t launch_batch_fused(int prec, int law, int mob, const void *inst, const int4 *work,
                               int nwork, int parity, int rows, int heun, const BatchNoise &nz,
                               cudaStream_t st);
cudaError_t launch_batch_diag(int prec, const void *inst, int first, int count, int blocks,
                              int parity, double *part, double *out, cudaStream_t st);
// nsteps steps of the work items [0, nwork) in one cooperative launch with
// a bounded grid barrier between steps; `barrier` is a device block of
// grid_barrier_bytes() whose first 8 bytes must be zero at launch and whose
// int at offset 8 becomes non-zero if a wait ran out.
size_t grid_barrier_bytes();
cudaError_t launch_batch_resident(int prec, int law, int mob, const void *inst, const int4 *work,
                                  int nwork, int parity, int rows, int nsteps, int heun,
                                  void *barrier, long long spin_limit, const BatchNoise &nz,
                                  cudaStream_t st);

}  // namespace cx

struct cx_ctx {
    cx_grid g;
    cx_params p;
    uint64_t seed;
    int prec;             // CX_PREC_*
    size_t elem;          // bytes per element
    long long pitch;      // elements per row (rows 128-byte aligned)
    void *b[2], *n[2];    // ping-pong state
    void *sigma;
    int own_fields;       // 1: b, n, sigma allocated (and freed) by the library
    int cur;              // index of the buffer holding the current state
    int64_t step;
    double dt;
    cudaStream_t stream;
    int device;
    int num_sms;          // streaming multiprocessors of that device
    int tile_rows;        // rows per step-kernel tile (0: automatic)
    int time_block;       // explicit stages per pass over the grid (1 or 2)
    cx::DiagScratch diag;
    double *h_diag;       // pinned [8]
    // staged uploads (cx_stage_state / cx_commit_state), created on first use
    void *stage_b, *stage_n;    // device staging arrays, library-owned, same pitch
    cudaStream_t copy_stream;   // the staged host-to-device copies
    cudaEvent_t staged;         // recorded after the staged copies
    cudaEvent_t stage_free;     // recorded once the compute stream is done with the staging arrays
    int stage_pending;          // a staged upload awaits cx_commit_state
    int stage_free_valid;       // stage_free has been recorded
};
