// cx_diag.cu -- diagnostics of the current state: dx^2 sum b, dx^2 sum n,
// the conserved combination dx^2 sum (b + theta n) (Eq. mass-conser and
// the no-flux walls of Eq. bconds), min/max, the envelope radius and a
// finiteness flag.
//
// Two kernels, both with a fixed launch shape so the summation order (and
// therefore the FP64 result) is the same on every call:
//   1. diag_partial (FP64 state) / diag_partial_f32 (FP32 state): block r
//      reduces rows r, r + G, r + 2G, ...; each thread accumulates its
//      columns (in FP64, or compensated FP32 flushed to FP64 once per row),
//      then warp shuffles and one shared-memory pass give one record per
//      block;
//   2. diag_final: one block folds the G block records in index order.
// The envelope radius is found exactly in integers: 4 r^2 / dx^2 =
// (2i+1-nx)^2 + (2j+1-ny)^2 for a cell centre.
#include <float.h>
#include <stdint.h>
#include <math.h>

#include "cx_internal.h"

namespace cx {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 1024;

struct Acc {
    double sb, sn;       // sums of b and n
    double mnb, mnn, mxb;
    long long r2;        // max (2i+1-nx)^2 + (2j+1-ny)^2 over b >= threshold, -1 if none
    int bad;             // count of non-finite cells (saturating flag)
};

__device__ __forceinline__ void combine(Acc &a, const Acc &o)
{
    a.sb += o.sb;
    a.sn += o.sn;
    a.mnb = fmin(a.mnb, o.mnb);
    a.mnn = fmin(a.mnn, o.mnn);
    a.mxb = fmax(a.mxb, o.mxb);
    a.r2 = max(a.r2, o.r2);
    a.bad |= o.bad;
}

__device__ __forceinline__ Acc shfl_down(const Acc &a, int d)
{
    Acc o;
    o.sb = __shfl_down_sync(0xffffffffu, a.sb, d);
    o.sn = __shfl_down_sync(0xffffffffu, a.sn, d);
    o.mnb = __shfl_down_sync(0xffffffffu, a.mnb, d);
    o.mnn = __shfl_down_sync(0xffffffffu, a.mnn, d);
    o.mxb = __shfl_down_sync(0xffffffffu, a.mxb, d);
    o.r2 = __shfl_down_sync(0xffffffffu, a.r2, d);
    o.bad = __shfl_down_sync(0xffffffffu, a.bad, d);
    return o;
}

__device__ __forceinline__ Acc empty_acc()
{
    Acc a;
    a.sb = 0.0; a.sn = 0.0;
    a.mnb = DBL_MAX; a.mnn = DBL_MAX; a.mxb = -DBL_MAX;
    a.r2 = -1; a.bad = 0;
    return a;
}

// Block-wide fold in a fixed order; the result is valid in thread 0.
__device__ Acc block_reduce(Acc a)
{
    __shared__ Acc warp_acc[kThreads / 32];
    for (int d = 16; d > 0; d >>= 1) combine(a, shfl_down(a, d));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) warp_acc[w] = a;
    __syncthreads();
    if (w == 0) {
        a = lane < kThreads / 32 ? warp_acc[lane] : empty_acc();
        for (int d = 16; d > 0; d >>= 1) combine(a, shfl_down(a, d));
    }
    return a;
}

__device__ __forceinline__ void store_acc(double *dst, const Acc &a)
{
    dst[0] = a.sb; dst[1] = a.sn; dst[2] = a.mnb; dst[3] = a.mnn; dst[4] = a.mxb;
    dst[5] = (double)a.r2;  // exact: below 2^53
    dst[6] = (double)a.bad;
    dst[7] = 0.0;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    diag_partial(const T *__restrict__ b, const T *__restrict__ n, int nx, int ny,
                 long long pitch, double bth, double *__restrict__ part)
{
    Acc a = empty_acc();
    for (int j = blockIdx.x; j < ny; j += gridDim.x) {
        const T *rb = b + (long long)j * pitch;
        const T *rn = n + (long long)j * pitch;
        const long long dy = 2LL * j + 1 - ny;
        for (int i = threadIdx.x; i < nx; i += kThreads) {
            const double vb = (double)rb[i], vn = (double)rn[i];
            a.sb += vb;
            a.sn += vn;
            if (!isfinite(vb) || !isfinite(vn)) a.bad = 1;
            a.mnb = fmin(a.mnb, vb);
            a.mnn = fmin(a.mnn, vn);
            a.mxb = fmax(a.mxb, vb);
            if (vb >= bth) {
                const long long ddx = 2LL * i + 1 - nx;
                a.r2 = max(a.r2, ddx * ddx + dy * dy);
            }
        }
    }
    a = block_reduce(a);
    if (threadIdx.x == 0) store_acc(part + 8LL * blockIdx.x, a);
}

// Knuth's error-free sum: s + c += x with s, c in FP32; (s, c) keeps the
// exact running total to O(len * eps^2).
__device__ __forceinline__ void two_sum(float &s, float &c, float x)
{
    const float t = s + x;
    const float z = t - s;
    c += (s - (t - z)) + (x - z);
    s = t;
}

// FP32 state: GB300's FP64 pipe is far slower than its FP32 pipe, so each
// thread sums its part of a row with compensated FP32 arithmetic and adds
// the (sum, error) pair to its FP64 totals once per row.  Minima and maxima
// are exact in FP32; `fth` is the least float f with (double)f >= b_th, so
// the threshold test decides exactly as an FP64 comparison would.  The
// envelope radius of a row is attained at its first or last column above
// the threshold ((2i+1-nx)^2 is convex in i).
template <bool VEC>
__global__ void __launch_bounds__(kThreads)
    diag_partial_f32(const float *__restrict__ b, const float *__restrict__ n, int nx, int ny,
                     long long pitch, float fth, double *__restrict__ part)
{
    double sb = 0.0, sn = 0.0;
    float mnb = FLT_MAX, mnn = FLT_MAX, mxb = -FLT_MAX;
    long long r2 = -1;
    int bad = 0;
    for (int j = blockIdx.x; j < ny; j += gridDim.x) {
        const float *rb = b + (long long)j * pitch;
        const float *rn = n + (long long)j * pitch;
        float bs = 0.f, bc = 0.f, ns = 0.f, nc = 0.f;
        int imin = 0x7fffffff, imax = -1;
        auto cell = [&](int i, float vb, float vn) {
            two_sum(bs, bc, vb);
            two_sum(ns, nc, vn);
            mnb = fminf(mnb, vb);
            mnn = fminf(mnn, vn);
            mxb = fmaxf(mxb, vb);
            bad |= !(isfinite(vb) && isfinite(vn));
            if (vb >= fth) {
                imin = min(imin, i);
                imax = max(imax, i);
            }
        };
        int tail = 0;
        if (VEC) {
            const int nv = nx >> 2;
            for (int v = threadIdx.x; v < nv; v += kThreads) {
                const float4 qb = __ldg(reinterpret_cast<const float4 *>(rb) + v);
                const float4 qn = __ldg(reinterpret_cast<const float4 *>(rn) + v);
                cell(4 * v, qb.x, qn.x);
                cell(4 * v + 1, qb.y, qn.y);
                cell(4 * v + 2, qb.z, qn.z);
                cell(4 * v + 3, qb.w, qn.w);
            }
            tail = nv << 2;
        }
        for (int i = tail + threadIdx.x; i < nx; i += kThreads) cell(i, rb[i], rn[i]);
        sb += (double)bs + (double)bc;
        sn += (double)ns + (double)nc;
        if (imax >= 0) {
            const long long d0 = 2LL * imin + 1 - nx, d1 = 2LL * imax + 1 - nx;
            const long long dy = 2LL * j + 1 - ny;
            r2 = max(r2, max(d0 * d0, d1 * d1) + dy * dy);
        }
    }
    Acc a;
    a.sb = sb; a.sn = sn;
    a.mnb = (double)mnb; a.mnn = (double)mnn; a.mxb = (double)mxb;
    a.r2 = r2; a.bad = bad;
    a = block_reduce(a);
    if (threadIdx.x == 0) store_acc(part + 8LL * blockIdx.x, a);
}

__global__ void __launch_bounds__(kThreads)
    diag_final(const double *__restrict__ part, int blocks, double *__restrict__ out)
{
    Acc a = empty_acc();
    for (int r = threadIdx.x; r < blocks; r += kThreads) {
        const double *p = part + 8LL * r;
        Acc o;
        o.sb = p[0]; o.sn = p[1]; o.mnb = p[2]; o.mnn = p[3]; o.mxb = p[4];
        o.r2 = (long long)p[5];
        o.bad = (int)p[6];
        combine(a, o);
    }
    a = block_reduce(a);
    if (threadIdx.x == 0) store_acc(out, a);
}

}  // namespace

int diag_blocks_for(int ny) { return ny < kMaxBlocks ? (ny < 1 ? 1 : ny) : kMaxBlocks; }

cudaError_t launch_diagnostics(int prec, const void *b, const void *n, int nx, int ny,
                               long long pitch, double b_threshold, DiagScratch s,
                               cudaStream_t st)
{
    if (prec == CX_PREC_F64) {
        diag_partial<double><<<s.blocks, kThreads, 0, st>>>((const double *)b, (const double *)n,
                                                            nx, ny, pitch, b_threshold, s.partials);
    } else {
        float fth = (float)b_threshold;
        if ((double)fth < b_threshold) fth = nextafterf(fth, INFINITY);
        const bool vec = (pitch % 4 == 0) && ((uintptr_t)b % 16 == 0) && ((uintptr_t)n % 16 == 0);
        if (vec)
            diag_partial_f32<true><<<s.blocks, kThreads, 0, st>>>((const float *)b, (const float *)n,
                                                                  nx, ny, pitch, fth, s.partials);
        else
            diag_partial_f32<false><<<s.blocks, kThreads, 0, st>>>(
                (const float *)b, (const float *)n, nx, ny, pitch, fth, s.partials);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    diag_final<<<1, kThreads, 0, st>>>(s.partials, s.blocks, s.result);
    return cudaGetLastError();
}

}  // namespace cx
