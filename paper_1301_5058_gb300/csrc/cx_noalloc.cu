// cx_noalloc.cu -- cx_diagnostics_noalloc: the diagnostics reduction over
// caller-owned fields with its scratch in a static device array, for callers
// that may not allocate (see include/cx.h).  The paper has no counterpart.
//
// The kernels are the ones cx_diagnostics launches (cx_diag.cu); only the
// home of their per-block partial records differs.  In host code the name
// g_diag_scratch is a host-side stand-in, not a device address, so the
// address is looked up with cudaGetSymbolAddress, with the device current,
// and passed to the launcher.  The lookup is cached per device and per CUDA
// context: a context that is destroyed and created again (cudaDeviceReset)
// loads the module again, possibly at another address, and gets a fresh
// lookup.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <cuda.h>
#include <mutex>

#include "cx_internal.h"

namespace {

constexpr int kScratchRecords = 1024;  // the reduction never uses more blocks
constexpr int kMaxDevices = 64;
// widest grid whose squared envelope radius (2i+1-nx)^2 + (2j+1-ny)^2 stays
// below 2^53, so that the record's slot 5 holds it exactly: (2^26)^2 = 2^52
// and, with ny <= 2,097,120 < 2^21, (2^21)^2 = 2^42
constexpr long long kMaxNx = 1LL << 26;

static __device__ __align__(256) double g_diag_scratch[kScratchRecords * 8];

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

struct Cached {
    unsigned long long ctx_id;  // 0: none
    void *addr;
};

std::mutex g_mu;
Cached g_cache[kMaxDevices] = {};
bool g_fns_tried = false;
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;

// The unique id of the current context (0 if there is none, or if the
// driver cannot tell: then nothing is cached).  Called with g_mu held.
unsigned long long current_ctx_id()
{
    if (!g_fns_tried) {
        g_fns_tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            g_ctx_current = (CtxGetCurrentFn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            g_ctx_id = (CtxGetIdFn)f;
        cudaGetLastError();
    }
    if (!g_ctx_current || !g_ctx_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (g_ctx_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

}  // namespace

// Record the failure for cx_last_error() and return its code.
static int noalloc_fail(int code, const char *msg, const char *detail)
{
    char buf[400];
    snprintf(buf, sizeof buf, "cx_diagnostics_noalloc: %s%s%s", msg, detail ? ": " : "",
             detail ? detail : "");
    return cx::record_error(code, buf);
}

// Device address of the scratch array in the current device's context.  The
// first call in a context looks it up (and, under lazy module loading, makes
// the driver load this file's module, which holds the array); later calls in
// the same context reuse it.
static int scratch_address(double **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(CX_ERR_CUDA, "cudaGetDevice", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(CX_ERR_CUDA, "device index out of range", nullptr);
    std::lock_guard<std::mutex> lock(g_mu);
    const unsigned long long id = current_ctx_id();
    if (id != 0 && g_cache[dev].ctx_id == id) {
        *out = (double *)g_cache[dev].addr;
        return CX_OK;
    }
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_diag_scratch);
    if (e != cudaSuccess || !p)
        return noalloc_fail(CX_ERR_CUDA, "cudaGetSymbolAddress", cudaGetErrorString(e));
    // the lookup made the device's primary context current if it was not
    g_cache[dev].ctx_id = current_ctx_id();
    g_cache[dev].addr = p;
    *out = (double *)p;
    return CX_OK;
}

extern "C" int cx_diagnostics_noalloc(const void *b, const void *n, int32_t nx, int32_t ny,
                                      int64_t pitch, int32_t precision, double dx, double theta,
                                      double b_threshold, void *stream, double *result_dev,
                                      cx_diag *out)
{
    if (!b || !n || !result_dev)
        return noalloc_fail(CX_ERR_INVALID_ARG, "b, n and result_dev must not be NULL", nullptr);
    if (nx < 1 || ny < 1 || pitch < nx)
        return noalloc_fail(CX_ERR_INVALID_ARG, "need nx, ny >= 1 and pitch >= nx", nullptr);
    if ((long long)nx * ny > (1LL << 32) || ny > 65535LL * 32 || nx > kMaxNx)
        return noalloc_fail(CX_ERR_INVALID_ARG,
                            "grid exceeds the maximum (nx*ny <= 2^32, nx <= 2^26, ny <= 2097120)",
                            nullptr);
    if (precision != CX_PREC_F64 && precision != CX_PREC_F32)
        return noalloc_fail(CX_ERR_INVALID_ARG, "precision must be CX_PREC_F64 or CX_PREC_F32", nullptr);
    if (!(isfinite(dx) && dx > 0.0) || !(isfinite(theta) && theta >= 0.0) ||
        !(isfinite(b_threshold) && b_threshold > 0.0))
        return noalloc_fail(CX_ERR_INVALID_ARG, "need dx > 0, theta >= 0, b_threshold > 0", nullptr);
    const int blocks = cx::diag_blocks_for(ny);
    if (blocks > kScratchRecords)
        return noalloc_fail(CX_ERR_INVALID_ARG, "reduction needs more partial records than the "
                                                "static scratch holds", nullptr);
    double *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    cx::DiagScratch s;
    s.partials = scratch;
    s.result = result_dev;
    s.blocks = blocks;
    cudaStream_t st = (cudaStream_t)stream;
    // the caller's fields are in natural in-row order
    cudaError_t e = cx::launch_diagnostics(precision, b, n, nx, ny, pitch, b_threshold, s, st, false);
    if (e != cudaSuccess) return noalloc_fail(CX_ERR_CUDA, "diagnostics launch", cudaGetErrorString(e));
    if (!out) return CX_OK;
    double h[8];
    e = cudaMemcpyAsync(h, result_dev, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return noalloc_fail(CX_ERR_CUDA, "result copy", cudaGetErrorString(e));
    const double area = dx * dx;
    memset(out, 0, sizeof *out);
    out->mass_b = area * h[0];
    out->mass_n = area * h[1];
    out->invariant = area * (h[0] + theta * h[1]);
    out->min_b = h[2];
    out->min_n = h[3];
    out->max_b = h[4];
    out->r_env = h[5] >= 0.0 ? 0.5 * dx * sqrt(h[5]) : 0.0;
    out->area_env = dx * dx * h[7];
    out->finite = h[6] == 0.0 ? 1 : 0;
    out->status = !out->finite ? CX_ERR_NONFINITE
                               : ((out->min_b < 0.0 || out->min_n < 0.0) ? CX_ERR_NEGATIVE : CX_OK);
    if (out->status != CX_OK)
        return noalloc_fail(out->status, out->status == CX_ERR_NONFINITE ? "non-finite value in the fields"
                                                                         : "negative density in the fields",
                            nullptr);
    return CX_OK;
}
