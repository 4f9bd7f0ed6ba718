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
//      block (cx_reduce.cuh);
//   2. diag_final: one block folds the G block records in index order.
// The envelope radius is found exactly in integers: 4 r^2 / dx^2 =
// (2i+1-nx)^2 + (2j+1-ny)^2 for a cell centre.
#include <math.h>

#include "cx_reduce.cuh"

namespace cx {
namespace {

using namespace reduce;

constexpr int kMaxBlocks = 1024;

template <bool PAIR>
__global__ void __launch_bounds__(kThreads)
    diag_partial(const double *__restrict__ b, const double *__restrict__ n, int nx, int ny,
                 long long pitch, double bth, double *__restrict__ part)
{
    Acc a = rows_f64<PAIR>(b, n, nx, ny, pitch, bth, blockIdx.x, gridDim.x);
    a = block_reduce(a);
    if (threadIdx.x == 0) store_acc(part + 8LL * blockIdx.x, a);
}

template <bool VEC, bool PAIR>
__global__ void __launch_bounds__(kThreads)
    diag_partial_f32(const float *__restrict__ b, const float *__restrict__ n, int nx, int ny,
                     long long pitch, float fth, double *__restrict__ part)
{
    Acc a = rows_f32<VEC, PAIR>(b, n, nx, ny, pitch, fth, blockIdx.x, gridDim.x);
    a = block_reduce(a);
    if (threadIdx.x == 0) store_acc(part + 8LL * blockIdx.x, a);
}

__global__ void __launch_bounds__(kThreads)
    diag_final(const double *__restrict__ part, int blocks, double *__restrict__ out)
{
    Acc a = empty_acc();
    for (int r = threadIdx.x; r < blocks; r += kThreads) combine(a, load_acc(part + 8LL * r));
    a = block_reduce(a);
    if (threadIdx.x == 0) store_acc(out, a);
}

}  // namespace

int diag_blocks_for(int ny) { return ny < kMaxBlocks ? (ny < 1 ? 1 : ny) : kMaxBlocks; }

cudaError_t launch_diagnostics(int prec, const void *b, const void *n, int nx, int ny,
                               long long pitch, double b_threshold, DiagScratch s,
                               cudaStream_t st, bool pair_order)
{
    if (prec == CX_PREC_F64) {
        if (pair_order)
            diag_partial<true><<<s.blocks, kThreads, 0, st>>>((const double *)b, (const double *)n,
                                                              nx, ny, pitch, b_threshold, s.partials);
        else
            diag_partial<false><<<s.blocks, kThreads, 0, st>>>((const double *)b, (const double *)n,
                                                               nx, ny, pitch, b_threshold, s.partials);
    } else {
        const float fth = float_threshold(b_threshold);
        const bool vec = (pitch % 4 == 0) && ((uintptr_t)b % 16 == 0) && ((uintptr_t)n % 16 == 0);
        const float *fb = (const float *)b, *fn = (const float *)n;
        if (pair_order)  // pair order implies rows of whole 16-byte groups
            diag_partial_f32<true, true><<<s.blocks, kThreads, 0, st>>>(fb, fn, nx, ny, pitch, fth,
                                                                        s.partials);
        else if (vec)
            diag_partial_f32<true, false><<<s.blocks, kThreads, 0, st>>>(fb, fn, nx, ny, pitch, fth,
                                                                         s.partials);
        else
            diag_partial_f32<false, false><<<s.blocks, kThreads, 0, st>>>(fb, fn, nx, ny, pitch,
                                                                          fth, s.partials);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    diag_final<<<1, kThreads, 0, st>>>(s.partials, s.blocks, s.result);
    return cudaGetLastError();
}

}  // namespace cx
