// cx_api.cu -- the C ABI declared in include/cx.h: parameter validation, the
// stability limit, buffer ownership, time stepping, diagnostics, field I/O
// and checkpoints.  Every step of the method runs in the library's kernels;
// this file only allocates, launches and copies.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "cx_internal.h"

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation)
        return fail(CX_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(CX_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CX_CUDA(call, what)                                     \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(e_, (what));    \
    } while (0)

bool finite_nonneg(double v) { return isfinite(v) && v >= 0.0; }

int validate(const cx_grid *g, const cx_params *p)
{
    if (!g || !p) return fail(CX_ERR_INVALID_ARG, "grid and params must not be NULL");
    if (g->nx < 1 || g->ny < 1)
        return fail(CX_ERR_INVALID_ARG, "grid %d x %d: both sides must be >= 1", g->nx, g->ny);
    if ((long long)g->nx * g->ny > (1LL << 32))
        return fail(CX_ERR_INVALID_ARG, "grid %d x %d exceeds 2^32 cells", g->nx, g->ny);
    if (g->ny > 65535LL * 32)
        return fail(CX_ERR_INVALID_ARG, "ny = %d exceeds %d", g->ny, 65535 * 32);
    if (!(isfinite(g->dx) && g->dx > 0.0))
        return fail(CX_ERR_INVALID_ARG, "dx must be finite and > 0");
    const struct { const char *name; double v; } nonneg[] = {
        {"n0", p->n0}, {"chi0", p->chi0}, {"sigma0", p->sigma0}, {"noise_amp", p->noise_amp},
        {"Dn", p->Dn}, {"theta", p->theta}, {"bM", p->bM}, {"dt", p->dt},
    };
    for (const auto &q : nonneg)
        if (!finite_nonneg(q.v))
            return fail(CX_ERR_INVALID_ARG, "%s = %g must be finite and >= 0", q.name, q.v);
    if (p->noise_amp > 1.0)
        return fail(CX_ERR_INVALID_ARG, "noise_amp = %g must be <= 1 (sigma >= 0)", p->noise_amp);
    if (!(isfinite(p->r0sq) && p->r0sq > 0.0))
        return fail(CX_ERR_INVALID_ARG, "r0sq must be finite and > 0");
    if (p->dt == 0.0 && !(isfinite(p->cfl_frac) && p->cfl_frac > 0.0 && p->cfl_frac <= 1.0))
        return fail(CX_ERR_INVALID_ARG, "cfl_frac = %g must lie in (0, 1]", p->cfl_frac);
    if (!isfinite(p->b_threshold))
        return fail(CX_ERR_INVALID_ARG, "b_threshold must be finite");
    if (p->chemo_law != CX_CHEMO_RECEPTOR && p->chemo_law != CX_CHEMO_CONSTANT)
        return fail(CX_ERR_INVALID_ARG, "chemo_law = %d", p->chemo_law);
    if (p->mobility != CX_MOBILITY_CENTRAL && p->mobility != CX_MOBILITY_UPWIND)
        return fail(CX_ERR_INVALID_ARG, "mobility = %d", p->mobility);
    if (p->noise_dist != CX_NOISE_UNIFORM && p->noise_dist != CX_NOISE_TRIANGULAR)
        return fail(CX_ERR_INVALID_ARG, "noise_dist = %d", p->noise_dist);
    if (p->noise_mode != CX_NOISE_STATIC && p->noise_mode != CX_NOISE_PER_STEP)
        return fail(CX_ERR_INVALID_ARG, "noise_mode = %d", p->noise_mode);
    if (p->scheme != CX_SCHEME_EULER && p->scheme != CX_SCHEME_HEUN)
        return fail(CX_ERR_INVALID_ARG, "scheme = %d", p->scheme);
    if (p->precision != CX_PREC_F64 && p->precision != CX_PREC_F32)
        return fail(CX_ERR_INVALID_ARG, "precision = %d", p->precision);
    return CX_OK;
}

double dt_limit_of(const cx_grid *g, const cx_params *p)
{
    const double B = p->bM + p->theta * p->n0;
    const double sigma_max = p->sigma0 * (1.0 + p->noise_amp);
    const double dchem = sigma_max * p->n0 * B * (1.0 + p->chi0 * B);
    const double dmax = p->Dn > dchem ? p->Dn : dchem;
    const double dx2 = g->dx * g->dx;
    const double l1 = dx2 / (4.0 * dmax);
    const double l2 = 1.0 / (4.0 * p->Dn / dx2 + B);
    return l1 < l2 ? l1 : l2;
}

double b_threshold_of(const cx_params *p)
{
    return p->b_threshold > 0.0 ? p->b_threshold : 0.1 * p->theta * p->n0;
}

int resolve_dt(const cx_grid *g, const cx_params *p, double *dt)
{
    const double lim = dt_limit_of(g, p);
    if (p->dt == 0.0) {
        *dt = p->cfl_frac * lim;
    } else {
        if (p->dt > lim)
            return fail(CX_ERR_DT_UNSTABLE, "dt = %.17g exceeds the stability limit %.17g", p->dt, lim);
        *dt = p->dt;
    }
    return CX_OK;
}

cx::Coef coef_of(const cx_ctx *c) { return cx::make_coef(c->g, c->p, c->dt); }

void free_buffers(cx_ctx *c)
{
    for (int q = 0; q < 2; ++q) {
        if (c->own_fields && c->b[q]) cudaFree(c->b[q]);
        if (c->own_fields && c->n[q]) cudaFree(c->n[q]);
        c->b[q] = c->n[q] = nullptr;
    }
    if (c->own_fields && c->sigma) cudaFree(c->sigma);
    if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
    if (c->stage_b) cudaFree(c->stage_b);
    if (c->stage_n) cudaFree(c->stage_n);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->staged) cudaEventDestroy(c->staged);
    if (c->stage_free) cudaEventDestroy(c->stage_free);
    c->stage_b = c->stage_n = nullptr;
    c->copy_stream = nullptr;
    c->staged = c->stage_free = nullptr;
    if (c->diag.partials) cudaFree(c->diag.partials);
    if (c->diag.result) cudaFree(c->diag.result);
    if (c->h_diag) cudaFreeHost(c->h_diag);
    c->sigma = nullptr;
    c->diag.partials = c->diag.result = nullptr;
    c->h_diag = nullptr;
}

// Device arrays a caller provides for the fields (cx_create_with_buffers).
struct FieldBuffers {
    void *b[2], *n[2], *sigma;
    long long pitch;  // elements per row
};

// Allocate the handle and its buffers, or adopt the caller's field arrays
// (contents: zero).
int alloc_ctx(const cx_grid *g, const cx_params *p, uint64_t seed, double dt, cx_ctx **out,
              const FieldBuffers *ext = nullptr)
{
    cx_ctx *c = new (std::nothrow) cx_ctx;
    if (!c) return fail(CX_ERR_OOM, "host allocation of the handle failed");
    memset(c, 0, sizeof *c);
    c->g = *g;
    c->p = *p;
    c->seed = seed;
    c->prec = p->precision;
    c->elem = c->prec == CX_PREC_F64 ? sizeof(double) : sizeof(float);
    const long long align = 128 / (long long)c->elem;  // rows start on 128-byte lines
    c->pitch = ext ? ext->pitch : ((long long)g->nx + align - 1) / align * align;
    c->own_fields = ext ? 0 : 1;
    c->dt = dt;
    c->tile_rows = 0;  // automatic (auto_tile_rows)
    // two stages per pass pay off for an FP32 state, whose pass is bound by
    // memory and instruction issue; the FP64 pass is bound by the FP64 pipe
    // and the fused pass's overlap lanes only add FP64 work
    c->time_block = c->prec == CX_PREC_F32 ? 2 : 1;
    c->stream = nullptr;
    cudaGetDevice(&c->device);
    c->num_sms = 0;
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess ||
        c->num_sms < 1) {
        cudaGetLastError();
        c->num_sms = 1;  // only the automatic tile height uses it
    }
    const size_t bytes = (size_t)c->pitch * (size_t)g->ny * c->elem;
    cudaError_t e = cudaSuccess;
    if (ext) {
        for (int q = 0; q < 2; ++q) {
            c->b[q] = ext->b[q];
            c->n[q] = ext->n[q];
        }
        c->sigma = ext->sigma;
    } else {
        for (int q = 0; q < 2 && e == cudaSuccess; ++q) {
            e = cudaMalloc(&c->b[q], bytes);
            if (e == cudaSuccess) e = cudaMalloc(&c->n[q], bytes);
        }
        if (e == cudaSuccess) e = cudaMalloc(&c->sigma, bytes);
    }
    c->diag.blocks = cx::diag_blocks_for(g->ny);
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->diag.partials, 8 * sizeof(double) * c->diag.blocks);
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->diag.result, 8 * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c->h_diag, 8 * sizeof(double));
    for (int q = 0; q < 2 && e == cudaSuccess; ++q) {
        e = cudaMemset(c->b[q], 0, bytes);
        if (e == cudaSuccess) e = cudaMemset(c->n[q], 0, bytes);
    }
    if (e == cudaSuccess) e = cudaMemset(c->sigma, 0, bytes);
    if (e != cudaSuccess) {
        free_buffers(c);
        delete c;
        cudaGetLastError();  // clear a sticky allocation error
        return cuda_fail(e, "device allocation");
    }
    *out = c;
    return CX_OK;
}

int check_ctx(const cx_ctx *c)
{
    if (!c) return fail(CX_ERR_INVALID_ARG, "NULL handle");
    return CX_OK;
}

void *field_ptr(cx_ctx *c, int which)
{
    if (which == CX_FIELD_B) return c->b[c->cur];
    if (which == CX_FIELD_N) return c->n[c->cur];
    return c->sigma;
}

// Which sigma recipe the handle uses: per-step noise of an FP32 state uses
// the FP32 recipe, everything else the FP64 one.
int sigma_recipe(const cx_ctx *c)
{
    return (c->p.noise_mode == CX_NOISE_PER_STEP && c->prec == CX_PREC_F32) ? 1 : 0;
}

// Write into the sigma array the field of time step `step` (per-step noise)
// or the static field (step 0).
cudaError_t fill_sigma(cx_ctx *c, int64_t step)
{
    return cx::launch_sigma_init(c->prec, c->sigma, c->g.nx, c->g.ny, c->pitch, c->seed,
                                 (uint64_t)step, c->p.sigma0, c->p.noise_amp, c->p.noise_dist,
                                 sigma_recipe(c), c->stream);
}

}  // namespace

int cx::record_error(int code, const char *msg) { return fail(code, "%s", msg); }
int cx::validate_params(const cx_grid *g, const cx_params *p) { return validate(g, p); }
int cx::resolve_time_step(const cx_grid *g, const cx_params *p, double *dt) { return resolve_dt(g, p, dt); }
double cx::envelope_level(const cx_params &p) { return b_threshold_of(&p); }
cx::Coef cx::make_coef(const cx_grid &g, const cx_params &p, double dt)
{
    const double dx2 = g.dx * g.dx;
    cx::Coef k;
    k.cA = dt / (8.0 * dx2);
    k.cChi = p.chemo_law == CX_CHEMO_RECEPTOR ? 2.0 * p.chi0 : 0.5 * p.chi0;
    k.cG = dt * p.Dn / dx2;
    k.cR = dt * p.theta;
    k.cN = dt;
    return k;
}

extern "C" {

int cx_version(void) { return CX_VERSION; }

const char *cx_strerror(int code)
{
    switch (code) {
    case CX_OK: return "ok";
    case CX_ERR_INVALID_ARG: return "invalid argument";
    case CX_ERR_DT_UNSTABLE: return "time step above the explicit stability limit";
    case CX_ERR_OOM: return "out of memory";
    case CX_ERR_CUDA: return "CUDA error";
    case CX_ERR_NONFINITE: return "non-finite value in the state";
    case CX_ERR_NEGATIVE: return "negative density in the state";
    case CX_ERR_TIMEOUT: return "device-side wait timed out";
    case CX_ERR_IO: return "checkpoint I/O error";
    case CX_ERR_UNSUPPORTED: return "unsupported option combination";
    default: return "unknown status code";
    }
}

const char *cx_last_error(void) { return g_err; }

int cx_params_default(cx_params *p)
{
    if (!p) return fail(CX_ERR_INVALID_ARG, "params must not be NULL");
    memset(p, 0, sizeof *p);
    p->n0 = 0.71;
    p->chi0 = 0.0;
    p->sigma0 = 1.0;
    p->noise_amp = 0.5;
    p->Dn = 1.0;
    p->theta = 1.0;
    p->bM = 0.71;
    p->r0sq = 6.25;
    p->dt = 0.0;
    p->cfl_frac = 0.2;
    p->b_threshold = 0.0;
    p->chemo_law = CX_CHEMO_RECEPTOR;
    p->mobility = CX_MOBILITY_CENTRAL;
    p->noise_dist = CX_NOISE_UNIFORM;
    p->noise_mode = CX_NOISE_STATIC;
    p->scheme = CX_SCHEME_EULER;
    p->precision = CX_PREC_F32;
    return CX_OK;
}

int cx_dt_limit(const cx_grid *g, const cx_params *p, double *limit)
{
    int rc = validate(g, p);
    if (rc) return rc;
    if (!limit) return fail(CX_ERR_INVALID_ARG, "limit must not be NULL");
    *limit = dt_limit_of(g, p);
    return CX_OK;
}

// Automatic tile height: 32 rows per tile for one stage per pass, 64 for two
// (the two-stage march's first and last tile rows repeat work of the
// neighbour tiles), or fewer so that a smaller grid still launches about four
// tiles per SM (eight with two stages, whose blocks hold fewer warps per SM)
// instead of a handful of long, latency-bound marches.
// Tall tiles amortise the halo rows a tile recomputes; enough tiles keep
// every SM busy on small grids.  Per SM: four 512-column CTAs (one stage
// per pass), sixteen 120-column one-warp CTAs (two stages, static sigma) or
// eight 480-column four-warp CTAs (two stages, sigma drawn per step).  On
// single FP32 grids with static sigma this picks 2, 4, 9 and 16 rows at
// sides 512, 1024, 1536 and 2048, the fastest measured heights or within
// 4 % of them (the earlier 480-column estimate picked 1, 3, 6 and 9 rows,
// 18-49 % slower), and 64 rows at 16384^2.
static int auto_tile_rows(const cx_ctx *c)
{
    const bool two = c->time_block == 2;
    const bool one_warp = two && c->p.noise_mode != CX_NOISE_PER_STEP;
    const long long cols = !two ? 512 : one_warp ? 120 : 480;
    const long long cap = two ? 64 : 32;
    const long long per_sm = !two ? 4 : one_warp ? 16 : 8;
    const long long tiles_x = ((long long)c->g.nx + cols - 1) / cols;
    const long long sms = c->num_sms;
    long long rows = ((long long)c->g.ny * tiles_x + per_sm * sms - 1) / (per_sm * sms);
    rows = rows < 1 ? 1 : (rows > cap ? cap : rows);
    while (((long long)c->g.ny + rows - 1) / rows > 65535) ++rows;
    return (int)rows;
}

static int tile_rows_of(const cx_ctx *c) { return c->tile_rows > 0 ? c->tile_rows : auto_tile_rows(c); }

static int create_ctx(const cx_grid *g, const cx_params *p, uint64_t seed, cx_ctx **out,
                      const FieldBuffers *ext)
{
    if (!out) return fail(CX_ERR_INVALID_ARG, "out must not be NULL");
    *out = nullptr;
    int rc = validate(g, p);
    if (rc) return rc;
    double dt;
    rc = resolve_dt(g, p, &dt);
    if (rc) return rc;
    cx_ctx *c;
    rc = alloc_ctx(g, p, seed, dt, &c, ext);
    if (rc) return rc;
    cudaError_t e = fill_sigma(c, 0);
    if (e == cudaSuccess)
        e = cx::launch_initial_state(c->prec, c->b[0], c->n[0], g->nx, g->ny, c->pitch, g->dx,
                                     p->n0, p->bM, p->r0sq, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cx_destroy(c);
        return cuda_fail(e, "initialisation kernels");
    }
    *out = c;
    return CX_OK;
}

int cx_create(const cx_grid *g, const cx_params *p, uint64_t seed, cx_ctx **out)
{
    return create_ctx(g, p, seed, out, nullptr);
}

int cx_create_with_buffers(const cx_grid *g, const cx_params *p, uint64_t seed, void *const b[2],
                           void *const n[2], void *sigma, int64_t pitch, cx_ctx **out)
{
    if (out) *out = nullptr;
    if (!b || !n) return fail(CX_ERR_INVALID_ARG, "b and n must point to two buffers each");
    int rc = validate(g, p);
    if (rc) return rc;
    FieldBuffers fb{{b[0], b[1]}, {n[0], n[1]}, sigma, (long long)pitch};
    const size_t elem = p->precision == CX_PREC_F64 ? sizeof(double) : sizeof(float);
    // rows hold whole groups of four cells (the pair order) in 16-byte units
    if (pitch < (int64_t)g->nx || pitch % 4 != 0 || ((size_t)pitch * elem) % 16 != 0)
        return fail(CX_ERR_INVALID_ARG, "pitch %lld: needs pitch >= nx = %d, a multiple of 4 "
                    "elements", (long long)pitch, g->nx);
    void *ptrs[5] = {fb.b[0], fb.b[1], fb.n[0], fb.n[1], fb.sigma};
    const unsigned long long span = (unsigned long long)pitch * (unsigned long long)g->ny * elem;
    for (int i = 0; i < 5; ++i) {
        if (!ptrs[i] || ((uintptr_t)ptrs[i] & 15) != 0)
            return fail(CX_ERR_INVALID_ARG, "field buffer %d is NULL or not 16-byte aligned", i);
        for (int j = 0; j < i; ++j) {
            const unsigned long long a = (uintptr_t)ptrs[i], q = (uintptr_t)ptrs[j];
            if (a < q + span && q < a + span)
                return fail(CX_ERR_INVALID_ARG, "field buffers %d and %d overlap", j, i);
        }
    }
    return create_ctx(g, p, seed, out, &fb);
}

int cx_set_stream(cx_ctx *c, void *stream)
{
    int rc = check_ctx(c);
    if (rc) return rc;
    c->stream = (cudaStream_t)stream;
    return CX_OK;
}

int cx_step(cx_ctx *c, int64_t n_steps)
{
    cx::NvtxRange range("cx_step");
    int rc = check_ctx(c);
    if (rc) return rc;
    if (n_steps < 0) return fail(CX_ERR_INVALID_ARG, "n_steps = %lld < 0", (long long)n_steps);
    cx::StepArgs a;
    a.nx = c->g.nx;
    a.ny = c->g.ny;
    a.pitch = c->pitch;
    a.law = c->p.chemo_law;
    a.mob = c->p.mobility;
    a.rows = tile_rows_of(c);
    a.k = coef_of(c);
    a.sg.per_step = c->p.noise_mode == CX_NOISE_PER_STEP;
    a.sg.dist = c->p.noise_dist;
    a.sg.sigma0 = c->p.sigma0;
    a.sg.amp = c->p.noise_amp;
    a.sg.seed = c->seed;
    a.s = c->sigma;
    const bool heun = c->p.scheme == CX_SCHEME_HEUN;
    int64_t m = 0;
    if (c->time_block == 2) {
        // two stages per pass: two Euler steps, or one whole Heun step
        const int64_t per_pass = heun ? 1 : 2;
        for (; m + per_pass <= n_steps; m += per_pass) {
            a.b = c->b[c->cur];
            a.n = c->n[c->cur];
            a.bu = a.nu = nullptr;
            a.bo = c->b[c->cur ^ 1];
            a.no = c->n[c->cur ^ 1];
            a.stage = 0;
            a.step = c->step;
            cudaError_t e = cx::launch_fused(c->prec, a, heun ? 1 : 0, c->stream);
            if (e != cudaSuccess) return cuda_fail(e, "fused step kernel launch");
            c->cur ^= 1;
            c->step += per_pass;
        }
    }
    for (; m < n_steps; ++m) {
        // Euler step, or Heun's first stage u* = u + dt r(u), into the other buffer
        a.b = c->b[c->cur];
        a.n = c->n[c->cur];
        a.bu = a.nu = nullptr;
        a.bo = c->b[c->cur ^ 1];
        a.no = c->n[c->cur ^ 1];
        a.stage = 0;
        a.step = c->step;
        cudaError_t e = cx::launch_step(c->prec, a, c->stream);
        if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
        if (heun) {
            // second stage: u' = (u + u* + dt r(u*)) / 2, written over u
            a.b = c->b[c->cur ^ 1];
            a.n = c->n[c->cur ^ 1];
            a.bu = c->b[c->cur];
            a.nu = c->n[c->cur];
            a.bo = c->b[c->cur];
            a.no = c->n[c->cur];
            a.stage = 1;
            e = cx::launch_step(c->prec, a, c->stream);
            if (e != cudaSuccess) return cuda_fail(e, "Heun stage launch");
        } else {
            c->cur ^= 1;
        }
        c->step += 1;
    }
    return CX_OK;
}

int cx_synchronize(cx_ctx *c)
{
    int rc = check_ctx(c);
    if (rc) return rc;
    CX_CUDA(cudaStreamSynchronize(c->stream), "stream synchronize");
    return CX_OK;
}

int cx_diagnostics(cx_ctx *c, cx_diag *out)
{
    cx::NvtxRange range("cx_diagnostics");
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!out) return fail(CX_ERR_INVALID_ARG, "out must not be NULL");
    const double bth = b_threshold_of(&c->p);
    CX_CUDA(cx::launch_diagnostics(c->prec, c->b[c->cur], c->n[c->cur], c->g.nx, c->g.ny,
                                   c->pitch, bth, c->diag, c->stream),
            "diagnostics launch");
    CX_CUDA(cudaMemcpyAsync(c->h_diag, c->diag.result, 8 * sizeof(double), cudaMemcpyDeviceToHost,
                            c->stream),
            "diagnostics copy");
    CX_CUDA(cudaStreamSynchronize(c->stream), "diagnostics synchronize");
    const double *h = c->h_diag;
    const double area = c->g.dx * c->g.dx;
    memset(out, 0, sizeof *out);
    out->step = c->step;
    out->dt = c->dt;
    out->t = (double)c->step * c->dt;
    out->mass_b = area * h[0];
    out->mass_n = area * h[1];
    out->invariant = area * (h[0] + c->p.theta * h[1]);
    out->min_b = h[2];
    out->min_n = h[3];
    out->max_b = h[4];
    out->r_env = h[5] >= 0.0 ? 0.5 * c->g.dx * sqrt(h[5]) : 0.0;
    out->area_env = c->g.dx * c->g.dx * h[7];
    out->finite = h[6] == 0.0 ? 1 : 0;
    out->status = CX_OK;
    if (!out->finite)
        out->status = CX_ERR_NONFINITE;
    else if (out->min_b < 0.0 || out->min_n < 0.0)
        out->status = CX_ERR_NEGATIVE;
    if (out->status != CX_OK)
        return fail(out->status, "state at step %lld: %s", (long long)c->step,
                    cx_strerror(out->status));
    return CX_OK;
}

static int check_io(cx_ctx *c, int32_t which, const void *host, int32_t dtype, size_t count)
{
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!host) return fail(CX_ERR_INVALID_ARG, "host pointer must not be NULL");
    if (which < CX_FIELD_B || which > CX_FIELD_SIGMA) return fail(CX_ERR_INVALID_ARG, "field %d", which);
    if (dtype != CX_F64 && dtype != CX_F32) return fail(CX_ERR_INVALID_ARG, "dtype %d", dtype);
    if (count != (size_t)c->g.nx * (size_t)c->g.ny)
        return fail(CX_ERR_INVALID_ARG, "count %zu != nx*ny = %zu", count,
                    (size_t)c->g.nx * (size_t)c->g.ny);
    return CX_OK;
}

// Rows of `row` bytes between a pitched and a packed array: one linear copy
// when the pitch equals the row (no padding), else a 2D copy.
static cudaError_t copy_rows(void *dst, size_t dpitch, const void *src, size_t spitch, size_t row,
                             size_t rows, cudaMemcpyKind kind, cudaStream_t st)
{
    if (dpitch == row && spitch == row) return cudaMemcpyAsync(dst, src, row * rows, kind, st);
    return cudaMemcpy2DAsync(dst, dpitch, src, spitch, row, rows, kind, st);
}

int cx_get_field(cx_ctx *c, int32_t which, void *host, int32_t dtype, size_t count)
{
    int rc = check_io(c, which, host, dtype, count);
    if (rc) return rc;
    const size_t row = (size_t)c->g.nx * c->elem;
    const int state_dtype = c->prec == CX_PREC_F64 ? CX_F64 : CX_F32;
    // with per-step noise, sigma is the field the next step will use
    if (which == CX_FIELD_SIGMA && c->p.noise_mode == CX_NOISE_PER_STEP)
        CX_CUDA(fill_sigma(c, c->step), "sigma regeneration");
    // the array in natural in-row order for the copy, and back afterwards
    void *f = field_ptr(c, which);
    CX_CUDA(cx::launch_pair_order(c->prec, f, c->g.nx, c->g.ny, c->pitch, c->stream), "reorder");
    if (dtype == state_dtype) {
        CX_CUDA(copy_rows(host, row, f, (size_t)c->pitch * c->elem, row, c->g.ny,
                          cudaMemcpyDeviceToHost, c->stream),
                "field copy to host");
        CX_CUDA(cx::launch_pair_order(c->prec, f, c->g.nx, c->g.ny, c->pitch, c->stream), "reorder");
        CX_CUDA(cudaStreamSynchronize(c->stream), "field copy synchronize");
        return CX_OK;
    }
    // precision change: copy in the state type, widen or narrow on the host
    std::vector<unsigned char> tmp;
    try { tmp.resize(count * c->elem); } catch (...) {
        cx::launch_pair_order(c->prec, f, c->g.nx, c->g.ny, c->pitch, c->stream);
        return fail(CX_ERR_OOM, "host staging");
    }
    CX_CUDA(copy_rows(tmp.data(), row, f, (size_t)c->pitch * c->elem, row, c->g.ny,
                      cudaMemcpyDeviceToHost, c->stream),
            "field copy to host");
    CX_CUDA(cx::launch_pair_order(c->prec, f, c->g.nx, c->g.ny, c->pitch, c->stream), "reorder");
    CX_CUDA(cudaStreamSynchronize(c->stream), "field copy synchronize");
    if (state_dtype == CX_F32) {
        const float *s = (const float *)tmp.data();
        double *d = (double *)host;
        for (size_t q = 0; q < count; ++q) d[q] = (double)s[q];
    } else {
        const double *s = (const double *)tmp.data();
        float *d = (float *)host;
        for (size_t q = 0; q < count; ++q) d[q] = (float)s[q];
    }
    return CX_OK;
}

int cx_set_field(cx_ctx *c, int32_t which, const void *host, int32_t dtype, size_t count)
{
    int rc = check_io(c, which, host, dtype, count);
    if (rc) return rc;
    if (which == CX_FIELD_SIGMA && c->p.noise_mode == CX_NOISE_PER_STEP)
        return fail(CX_ERR_INVALID_ARG, "sigma is regenerated every step with per-step noise");
    const size_t row = (size_t)c->g.nx * c->elem;
    const int state_dtype = c->prec == CX_PREC_F64 ? CX_F64 : CX_F32;
    CX_CUDA(cudaStreamSynchronize(c->stream), "synchronize before field write");
    const void *src = host;
    std::vector<unsigned char> tmp;
    if (dtype != state_dtype) {
        try { tmp.resize(count * c->elem); } catch (...) { return fail(CX_ERR_OOM, "host staging"); }
        if (state_dtype == CX_F32) {
            const double *s = (const double *)host;
            float *d = (float *)tmp.data();
            for (size_t q = 0; q < count; ++q) d[q] = (float)s[q];
        } else {
            const float *s = (const float *)host;
            double *d = (double *)tmp.data();
            for (size_t q = 0; q < count; ++q) d[q] = (double)s[q];
        }
        src = tmp.data();
    }
    CX_CUDA(copy_rows(field_ptr(c, which), (size_t)c->pitch * c->elem, src, row, row, c->g.ny,
                      cudaMemcpyHostToDevice, c->stream),
            "field copy to device");
    CX_CUDA(cx::launch_pair_order(c->prec, field_ptr(c, which), c->g.nx, c->g.ny, c->pitch,
                                  c->stream),
            "reorder");
    CX_CUDA(cudaStreamSynchronize(c->stream), "field copy synchronize");
    return CX_OK;
}

int cx_stage_state(cx_ctx *c, const void *b_host, const void *n_host, int32_t dtype, size_t count)
{
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!b_host || !n_host) return fail(CX_ERR_INVALID_ARG, "host pointers must not be NULL");
    const int state_dtype = c->prec == CX_PREC_F64 ? CX_F64 : CX_F32;
    if (dtype != state_dtype)
        return fail(CX_ERR_INVALID_ARG, "staged uploads take the state's own type (dtype %d)", state_dtype);
    if (count != (size_t)c->g.nx * (size_t)c->g.ny)
        return fail(CX_ERR_INVALID_ARG, "count %zu != nx*ny = %zu", count,
                    (size_t)c->g.nx * (size_t)c->g.ny);
    if (c->stage_pending)
        return fail(CX_ERR_INVALID_ARG, "an upload is already staged: commit it first");
    const size_t bytes = (size_t)c->pitch * (size_t)c->g.ny * c->elem;
    if (!c->copy_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->staged, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->stage_free, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(&c->stage_b, bytes);
        if (e == cudaSuccess) e = cudaMalloc(&c->stage_n, bytes);
        if (e == cudaSuccess && c->pitch != c->g.nx) {
            // the padding columns stay zero, as in the state arrays
            e = cudaMemsetAsync(c->stage_b, 0, bytes, c->copy_stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(c->stage_n, 0, bytes, c->copy_stream);
        }
        if (e != cudaSuccess) {
            if (c->stage_b) cudaFree(c->stage_b);
            if (c->stage_n) cudaFree(c->stage_n);
            if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
            if (c->staged) cudaEventDestroy(c->staged);
            if (c->stage_free) cudaEventDestroy(c->stage_free);
            c->stage_b = c->stage_n = nullptr;
            c->copy_stream = nullptr;
            c->staged = c->stage_free = nullptr;
            cudaGetLastError();
            return cuda_fail(e, "staging buffers");
        }
    }
    // the staging arrays may still be read by work queued before the last commit
    if (c->stage_free_valid) CX_CUDA(cudaStreamWaitEvent(c->copy_stream, c->stage_free, 0), "stage wait");
    const size_t row = (size_t)c->g.nx * c->elem;
    CX_CUDA(copy_rows(c->stage_b, (size_t)c->pitch * c->elem, b_host, row, row, c->g.ny,
                      cudaMemcpyHostToDevice, c->copy_stream),
            "staged copy of b");
    CX_CUDA(copy_rows(c->stage_n, (size_t)c->pitch * c->elem, n_host, row, row, c->g.ny,
                      cudaMemcpyHostToDevice, c->copy_stream),
            "staged copy of n");
    // into the pair order of the state arrays, still on the copy stream
    CX_CUDA(cx::launch_pair_order(c->prec, c->stage_b, c->g.nx, c->g.ny, c->pitch, c->copy_stream),
            "staged reorder of b");
    CX_CUDA(cx::launch_pair_order(c->prec, c->stage_n, c->g.nx, c->g.ny, c->pitch, c->copy_stream),
            "staged reorder of n");
    CX_CUDA(cudaEventRecord(c->staged, c->copy_stream), "stage event");
    c->stage_pending = 1;
    return CX_OK;
}

int cx_commit_state(cx_ctx *c)
{
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!c->stage_pending) return fail(CX_ERR_INVALID_ARG, "no upload is staged");
    CX_CUDA(cudaStreamWaitEvent(c->stream, c->staged, 0), "commit wait");
    if (c->own_fields) {
        // the staged arrays become the current state; the old current
        // arrays become the staging arrays once the queued work is done
        void *t = c->b[c->cur];
        c->b[c->cur] = c->stage_b;
        c->stage_b = t;
        t = c->n[c->cur];
        c->n[c->cur] = c->stage_n;
        c->stage_n = t;
    } else {
        // caller-owned state arrays keep their addresses: copy on the device
        // (whole groups of four: a row's last cell may lie in the padding)
        const size_t row = (size_t)((c->g.nx + 3) & ~3) * c->elem, pitch = (size_t)c->pitch * c->elem;
        CX_CUDA(copy_rows(c->b[c->cur], pitch, c->stage_b, pitch, row, c->g.ny,
                          cudaMemcpyDeviceToDevice, c->stream),
                "commit copy of b");
        CX_CUDA(copy_rows(c->n[c->cur], pitch, c->stage_n, pitch, row, c->g.ny,
                          cudaMemcpyDeviceToDevice, c->stream),
                "commit copy of n");
    }
    CX_CUDA(cudaEventRecord(c->stage_free, c->stream), "commit event");
    c->stage_free_valid = 1;
    c->stage_pending = 0;
    return CX_OK;
}

int cx_polar_profile(cx_ctx *c, double radius, int32_t nsamples, double *host_out)
{
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!host_out || nsamples < 1 || nsamples > (1 << 24) || !(isfinite(radius) && radius >= 0.0))
        return fail(CX_ERR_INVALID_ARG, "need host_out, 1 <= nsamples <= 2^24, radius >= 0");
    double *d = nullptr;
    CX_CUDA(cudaMalloc((void **)&d, sizeof(double) * (size_t)nsamples), "profile buffer");
    cudaError_t e = cx::launch_polar(c->prec, c->b[c->cur], c->g.nx, c->g.ny, c->pitch, c->g.dx,
                                     radius, nsamples, d, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host_out, d, sizeof(double) * (size_t)nsamples, cudaMemcpyDeviceToHost,
                            c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "polar profile");
    return CX_OK;
}

int cx_get_config(cx_ctx *c, cx_grid *g, cx_params *p, uint64_t *seed)
{
    int rc = check_ctx(c);
    if (rc) return rc;
    if (g) *g = c->g;
    if (p) {
        *p = c->p;
        p->dt = c->dt;
    }
    if (seed) *seed = c->seed;
    return CX_OK;
}

int cx_get_time(cx_ctx *c, int64_t *step, double *t, double *dt)
{
    int rc = check_ctx(c);
    if (rc) return rc;
    if (step) *step = c->step;
    if (t) *t = (double)c->step * c->dt;
    if (dt) *dt = c->dt;
    return CX_OK;
}

int cx_set_step(cx_ctx *c, int64_t step)
{
    int rc = check_ctx(c);
    if (rc) return rc;
    if (step < 0) return fail(CX_ERR_INVALID_ARG, "step = %lld < 0", (long long)step);
    c->step = step;
    return CX_OK;
}

int cx_set_tile_rows(cx_ctx *c, int32_t rows)
{
    int rc = check_ctx(c);
    if (rc) return rc;
    if (rows == 0) {  // back to the automatic height
        c->tile_rows = 0;
        return CX_OK;
    }
    if (rows < 1 || rows > 4096 || ((long long)c->g.ny + rows - 1) / rows > 65535)
        return fail(CX_ERR_INVALID_ARG, "tile rows %d outside 1..4096 or too small for ny = %d",
                    rows, c->g.ny);
    c->tile_rows = rows;
    return CX_OK;
}

int cx_get_tile_rows(cx_ctx *c, int32_t *rows)
{
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!rows) return fail(CX_ERR_INVALID_ARG, "rows must not be NULL");
    *rows = tile_rows_of(c);
    return CX_OK;
}

int cx_set_time_block(cx_ctx *c, int32_t stages)
{
    int rc = check_ctx(c);
    if (rc) return rc;
    if (stages != 1 && stages != 2)
        return fail(CX_ERR_INVALID_ARG, "time block %d: must be 1 or 2 stages per pass", stages);
    c->time_block = stages;
    return CX_OK;
}

int cx_get_time_block(cx_ctx *c, int32_t *stages)
{
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!stages) return fail(CX_ERR_INVALID_ARG, "stages must not be NULL");
    *stages = c->time_block;
    return CX_OK;
}

// Checkpoint layout (little-endian host order):
//   char magic[8] = "CXCKPT01"; cx_grid; cx_params; uint64 seed; int64 step;
//   double dt; int32 precision; int32 reserved;
//   then b, n, sigma as nx*ny elements each in the state precision.
static const char kMagic[8] = {'C', 'X', 'C', 'K', 'P', 'T', '0', '1'};

int cx_save(cx_ctx *c, const char *path)
{
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!path) return fail(CX_ERR_INVALID_ARG, "path must not be NULL");
    const size_t count = (size_t)c->g.nx * (size_t)c->g.ny;
    std::vector<unsigned char> buf;
    try { buf.resize(count * c->elem); } catch (...) { return fail(CX_ERR_OOM, "host staging"); }
    FILE *f = fopen(path, "wb");
    if (!f) return fail(CX_ERR_IO, "cannot open %s for writing", path);
    const int32_t prec = c->prec, reserved = 0;
    bool ok = fwrite(kMagic, 1, 8, f) == 8 && fwrite(&c->g, sizeof c->g, 1, f) == 1 &&
              fwrite(&c->p, sizeof c->p, 1, f) == 1 && fwrite(&c->seed, 8, 1, f) == 1 &&
              fwrite(&c->step, 8, 1, f) == 1 && fwrite(&c->dt, 8, 1, f) == 1 &&
              fwrite(&prec, 4, 1, f) == 1 && fwrite(&reserved, 4, 1, f) == 1;
    const int dtype = c->prec == CX_PREC_F64 ? CX_F64 : CX_F32;
    for (int w = CX_FIELD_B; ok && w <= CX_FIELD_SIGMA; ++w) {
        rc = cx_get_field(c, w, buf.data(), dtype, count);
        if (rc) { fclose(f); return rc; }
        ok = fwrite(buf.data(), c->elem, count, f) == count;
    }
    if (fclose(f) != 0) ok = false;
    if (!ok) return fail(CX_ERR_IO, "short write to %s", path);
    return CX_OK;
}

int cx_load(const char *path, cx_ctx **out)
{
    if (!out) return fail(CX_ERR_INVALID_ARG, "out must not be NULL");
    *out = nullptr;
    if (!path) return fail(CX_ERR_INVALID_ARG, "path must not be NULL");
    FILE *f = fopen(path, "rb");
    if (!f) return fail(CX_ERR_IO, "cannot open %s", path);
    char magic[8];
    cx_grid g;
    cx_params p;
    uint64_t seed;
    int64_t step;
    double dt;
    int32_t prec, reserved;
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kMagic, 8) == 0 &&
              fread(&g, sizeof g, 1, f) == 1 && fread(&p, sizeof p, 1, f) == 1 &&
              fread(&seed, 8, 1, f) == 1 && fread(&step, 8, 1, f) == 1 &&
              fread(&dt, 8, 1, f) == 1 && fread(&prec, 4, 1, f) == 1 &&
              fread(&reserved, 4, 1, f) == 1;
    if (!ok || prec != p.precision) {
        fclose(f);
        return fail(CX_ERR_IO, "%s is not a checkpoint of this library", path);
    }
    int rc = validate(&g, &p);
    if (rc) { fclose(f); return rc; }
    if (!(isfinite(dt) && dt > 0.0) || step < 0) {
        fclose(f);
        return fail(CX_ERR_IO, "%s: bad time step or step count", path);
    }
    cx_ctx *c;
    rc = alloc_ctx(&g, &p, seed, dt, &c);
    if (rc) { fclose(f); return rc; }
    c->step = step;
    const size_t count = (size_t)g.nx * (size_t)g.ny;
    std::vector<unsigned char> buf;
    try { buf.resize(count * c->elem); } catch (...) { fclose(f); cx_destroy(c); return fail(CX_ERR_OOM, "host staging"); }
    const int dtype = c->prec == CX_PREC_F64 ? CX_F64 : CX_F32;
    for (int w = CX_FIELD_B; w <= CX_FIELD_SIGMA; ++w) {
        if (fread(buf.data(), c->elem, count, f) != count) {
            fclose(f);
            cx_destroy(c);
            return fail(CX_ERR_IO, "%s is truncated", path);
        }
        // sigma is written even for per-step noise (it is then regenerated)
        if (w == CX_FIELD_SIGMA && p.noise_mode == CX_NOISE_PER_STEP) continue;
        rc = cx_set_field(c, w, buf.data(), dtype, count);
        if (rc) { fclose(f); cx_destroy(c); return rc; }
    }
    fclose(f);
    *out = c;
    return CX_OK;
}

void cx_destroy(cx_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    free_buffers(c);
    delete c;
}

}  // extern "C"
