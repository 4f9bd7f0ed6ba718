// cx_reduce.cuh -- the diagnostics reduction shared by the single-grid and
// batched diagnostics kernels: one record per thread / warp / block with
// the sums of b and n, min b, min n, max b, the largest
// (2i+1-nx)^2 + (2j+1-ny)^2 over cells with b >= b_th, a non-finite flag and
// the number of cells with b >= b_th.
#pragma once

#include <float.h>
#include <stdint.h>

#include "cx_internal.h"

namespace cx {
namespace reduce {

constexpr int kThreads = 256;

struct Acc {
    double sb, sn;  // sums of b and n
    double mnb, mnn, mxb;
    long long r2;   // max (2i+1-nx)^2 + (2j+1-ny)^2 over b >= threshold, -1 if none
    int bad;        // 1 if a non-finite cell was seen
    long long cnt;  // cells with b >= threshold
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
    a.cnt += o.cnt;
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
    o.cnt = __shfl_down_sync(0xffffffffu, a.cnt, d);
    return o;
}

__device__ __forceinline__ Acc empty_acc()
{
    Acc a;
    a.sb = 0.0; a.sn = 0.0;
    a.mnb = DBL_MAX; a.mnn = DBL_MAX; a.mxb = -DBL_MAX;
    a.r2 = -1; a.bad = 0; a.cnt = 0;
    return a;
}

// Block-wide fold in a fixed order (blockDim.x == kThreads); the result is
// valid in thread 0.
__device__ __forceinline__ Acc block_reduce(Acc a)
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
    // exact while r2 < 2^53, i.e. for nx <= 2^26 (ny is at most 2,097,120);
    // a wider grid rounds it to the nearest double, a relative change below
    // 2^-53 (no overflow: |2i+1-nx| < 2^31)
    dst[5] = (double)a.r2;
    dst[6] = (double)a.bad;
    dst[7] = (double)a.cnt;  // exact: at most 2^32 cells
}

__device__ __forceinline__ Acc load_acc(const double *p)
{
    Acc o;
    o.sb = p[0]; o.sn = p[1]; o.mnb = p[2]; o.mnn = p[3]; o.mxb = p[4];
    o.r2 = (long long)p[5];
    o.bad = (int)p[6];
    o.cnt = (long long)p[7];
    return o;
}

// FP64 state: rows j = j0, j0 + jstep, ... of one grid, this thread's
// elements.  PAIR: the rows are in the library's pair order (cx_internal.h),
// so the element at position p of a row is the cell in column pair_col(p).
template <bool PAIR>
__device__ __forceinline__ Acc rows_f64(const double *__restrict__ b, const double *__restrict__ n,
                                        int nx, int ny, long long pitch, double bth, int j0,
                                        int jstep)
{
    Acc a = empty_acc();
    const int width = PAIR ? (nx + 3) & ~3 : nx;
    for (int j = j0; j < ny; j += jstep) {
        const double *rb = b + (long long)j * pitch;
        const double *rn = n + (long long)j * pitch;
        const long long dy = 2LL * j + 1 - ny;
        for (int p = threadIdx.x; p < width; p += kThreads) {
            const int i = PAIR ? (int)pair_col(p) : p;
            if (PAIR && i >= nx) continue;
            const double vb = rb[p], vn = rn[p];
            a.sb += vb;
            a.sn += vn;
            if (!isfinite(vb) || !isfinite(vn)) a.bad = 1;
            a.mnb = fmin(a.mnb, vb);
            a.mnn = fmin(a.mnn, vn);
            a.mxb = fmax(a.mxb, vb);
            if (vb >= bth) {
                const long long ddx = 2LL * i + 1 - nx;
                a.r2 = max(a.r2, ddx * ddx + dy * dy);
                ++a.cnt;
            }
        }
    }
    return a;
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
// the threshold ((2i+1-nx)^2 is convex in i).  VEC: rows start 16-byte
// aligned, so whole float4 vectors are read.  PAIR: the rows are in the
// library's pair order (a vector holds columns 4v, 4v+2, 4v+1, 4v+3).
template <bool VEC, bool PAIR>
__device__ __forceinline__ Acc rows_f32(const float *__restrict__ b, const float *__restrict__ n,
                                        int nx, int ny, long long pitch, float fth, int j0,
                                        int jstep)
{
    double sb = 0.0, sn = 0.0;
    float mnb = FLT_MAX, mnn = FLT_MAX, mxb = -FLT_MAX;
    long long r2 = -1, cnt = 0;
    int bad = 0;
    for (int j = j0; j < ny; j += jstep) {
        const float *rb = b + (long long)j * pitch;
        const float *rn = n + (long long)j * pitch;
        float bs = 0.f, bc = 0.f, ns = 0.f, nc = 0.f;
        int imin = 0x7fffffff, imax = -1, above = 0;
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
                ++above;
            }
        };
        int tail = 0;
        if (VEC) {
            const int nv = nx >> 2;
            for (int v = threadIdx.x; v < nv; v += kThreads) {
                const float4 qb = __ldg(reinterpret_cast<const float4 *>(rb) + v);
                const float4 qn = __ldg(reinterpret_cast<const float4 *>(rn) + v);
                cell(4 * v, qb.x, qn.x);
                cell(4 * v + (PAIR ? 2 : 1), qb.y, qn.y);
                cell(4 * v + (PAIR ? 1 : 2), qb.z, qn.z);
                cell(4 * v + 3, qb.w, qn.w);
            }
            tail = nv << 2;
        }
        if (PAIR) {
            const int width = (nx + 3) & ~3;
            for (int p = tail + threadIdx.x; p < width; p += kThreads) {
                const int i = (int)pair_col(p);
                if (i < nx) cell(i, rb[p], rn[p]);
            }
        } else {
            for (int i = tail + threadIdx.x; i < nx; i += kThreads) cell(i, rb[i], rn[i]);
        }
        cnt += above;
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
    a.r2 = r2; a.bad = bad; a.cnt = cnt;
    return a;
}

// The least float f with (double)f >= t.
inline float float_threshold(double t)
{
    float f = (float)t;
    if ((double)f < t) f = nextafterf(f, INFINITY);
    return f;
}

}  // namespace reduce
}  // namespace cx
