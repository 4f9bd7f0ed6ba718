// cx_init.cu -- sigma field and initial state.
//
// sigma = sigma0 (1 + a Delta) (Eq. CoefCrsDif) with Delta drawn per cell
// from Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11), counter (cell index lo, hi, time
// step lo, hi) -- or (cell index / 4, step) for the FP32 recipe -- key
// (seed lo, hi).  Delta is formed exactly in integers and
// the products are rounded one at a time (no fused multiply-add), so the
// field is bit-identical to any other IEEE implementation of the same
// definition.  Two recipes exist (cx_philox.cuh): the FP64 one (static
// noise in either precision, and per-step noise of an FP64 state) and the
// FP32 one (per-step noise of an FP32 state).
//
// Initial state (Eq. inicond, Eq. inibacexp): n = n0, b = bM exp(-r^2/r0sq)
// with r the distance of the cell centre from the domain centre, cut to
// zero where r^2/r0sq > 40.  Both write the arrays in pair order
// (cx_internal.h), as do the step kernels; launch_pair_order converts an
// array between that order and the natural one.
#include "cx_internal.h"
#include "cx_philox.cuh"

namespace cx {
namespace {

template <typename T>
__global__ void sigma_init_kernel(T *__restrict__ sigma, int nx, int ny, long long pitch,
                                  uint64_t seed, uint64_t step, double sigma0, double amp,
                                  int dist, int recipe)
{
    const long long total = (long long)nx * ny;
    const float s0f = (float)sigma0, af = (float)amp;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < total;
         c += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(c / nx), i = (int)(c - (long long)j * nx);
        T v;
        if (recipe == 0)
            v = (T)sigma_f64(seed, (uint64_t)c, step, dist, sigma0, amp);
        else
            v = (T)sigma_f32(seed, (uint64_t)c, step, dist, s0f, af);
        sigma[(long long)j * pitch + pair_col(i)] = v;
    }
}

template <typename T>
__global__ void initial_state_kernel(T *__restrict__ b, T *__restrict__ n, int nx, int ny,
                                     long long pitch, double dx, double n0, double bM,
                                     double r0sq)
{
    const long long total = (long long)nx * ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < total;
         c += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(c / nx), i = (int)(c - (long long)j * nx);
        // (i + 1/2 - nx/2) is a half-integer: exact in FP64
        const double x = __dmul_rn((double)i + 0.5 - 0.5 * (double)nx, dx);
        const double y = __dmul_rn((double)j + 0.5 - 0.5 * (double)ny, dx);
        const double r2 = __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y));
        const double q = __ddiv_rn(-r2, r0sq);
        // the inoculum is cut to zero where r^2 / r0sq > 40 (compact support:
        // an FP32 and an FP64 state start alike; the mass changes by less
        // than e^-40), which also spares the exp of most cells of a grid
        const double e = q < -40.0 ? 0.0 : exp(q);
        b[(long long)j * pitch + pair_col(i)] = (T)__dmul_rn(bM, e);
        n[(long long)j * pitch + pair_col(i)] = (T)n0;
    }
}

// Swap the middle two elements of every group of four, for the groups that
// hold the row's nx cells.
template <typename T>
__global__ void pair_order_kernel(T *__restrict__ a, int groups, int ny, long long pitch)
{
    const long long total = (long long)groups * ny;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const long long j = q / groups, g = q - j * groups;
        T *p = a + j * pitch + 4 * g;
        const T x = p[1];
        p[1] = p[2];
        p[2] = x;
    }
}

int grid_for(long long total, int threads)
{
    long long g = (total + threads - 1) / threads;
    return (int)(g < 152LL * 32 ? (g < 1 ? 1 : g) : 152LL * 32);
}

}  // namespace

cudaError_t launch_sigma_init(int prec, void *sigma, int nx, int ny, long long pitch,
                              uint64_t seed, uint64_t step, double sigma0, double amp,
                              int dist, int recipe, cudaStream_t st)
{
    const int threads = 256;
    const int grid = grid_for((long long)nx * ny, threads);
    if (prec == CX_PREC_F64)
        sigma_init_kernel<double><<<grid, threads, 0, st>>>((double *)sigma, nx, ny, pitch, seed,
                                                            step, sigma0, amp, dist, recipe);
    else
        sigma_init_kernel<float><<<grid, threads, 0, st>>>((float *)sigma, nx, ny, pitch, seed,
                                                           step, sigma0, amp, dist, recipe);
    return cudaGetLastError();
}

cudaError_t launch_pair_order(int prec, void *a, int nx, int ny, long long pitch, cudaStream_t st)
{
    const int groups = (nx + 3) / 4;
    const int threads = 256;
    const int grid = grid_for((long long)groups * ny, threads);
    if (prec == CX_PREC_F64)
        pair_order_kernel<double><<<grid, threads, 0, st>>>((double *)a, groups, ny, pitch);
    else
        pair_order_kernel<float><<<grid, threads, 0, st>>>((float *)a, groups, ny, pitch);
    return cudaGetLastError();
}

cudaError_t launch_initial_state(int prec, void *b, void *n, int nx, int ny, long long pitch,
                                 double dx, double n0, double bM, double r0sq, cudaStream_t st)
{
    const int threads = 256;
    const int grid = grid_for((long long)nx * ny, threads);
    if (prec == CX_PREC_F64)
        initial_state_kernel<double><<<grid, threads, 0, st>>>((double *)b, (double *)n, nx, ny,
                                                               pitch, dx, n0, bM, r0sq);
    else
        initial_state_kernel<float><<<grid, threads, 0, st>>>((float *)b, (float *)n, nx, ny,
                                                              pitch, dx, n0, bM, r0sq);
    return cudaGetLastError();
}

}  // namespace cx
