// cx_batch.cu -- many independent simulations stepped together: parameter
// sweeps over (n0, chi0, sigma0) on grids of different sizes.
//
// Layout: one device arena holds every instance's b[2], n[2] and sigma
// (rows 128-byte aligned, arrays 256-byte aligned).  A device table holds
// each instance's pointers, size and flux coefficients; a work list holds
// one entry (instance, tile x, tile y) per 512-column x `rows`-row tile,
// instance by instance.  One launch of batch_step_kernel advances every
// tile of a range of instances by one step: the kernel boundary is the only
// barrier, so no block ever waits on another.  Runs of steps are captured
// once into a CUDA graph and replayed.  With a group size set, instances are
// cut into consecutive groups whose fields fit that many bytes (e.g. L2) and
// each group runs all its steps before the next starts.
//
// With two stages per pass (batch_fused_kernel) a second work list holds
// one entry per 120-column x `rows`-row tile (one warp) of the two-stage
// march.
//
// Every instance goes through the same per-thread stencil code as a single
// grid (cx_stencil.cuh, cx_fused.cuh), so a batch instance and a cx_ctx with
// the same grid, parameters and seed give bit-identical fields.
//
// This file holds the diagnostics kernels and the dispatch; the step kernels
// are in cx_batch_kernels.cuh, instantiated by cx_batch_inst.cu.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "cx_reduce.cuh"
#include "cx_batch_types.cuh"

namespace cx {
namespace batch {
// defined in cx_batch_kernels.cuh, instantiated in cx_batch_inst.cu
template <typename T, int LAW, int MOB>
cudaError_t launch_step_lm(const void *inst, const int4 *work, int nwork, int parity, int rows,
                           int stage, int noise, const long long *step_base, int step_off,
                           cudaStream_t st);
template <typename T, int LAW, int MOB>
cudaError_t launch_fused_lm(const void *inst, const int4 *work, int nwork, int parity, int rows,
                            int heun, int noise, const long long *step_base, int step_off,
                            cudaStream_t st);
template <typename T, int LAW, int MOB>
cudaError_t launch_resident_lm(const void *inst, const int4 *work, int nwork, int parity,
                               int rows, int nsteps, int heun, int noise, void *gb,
                               long long spin, const long long *step_base, int step_off,
                               cudaStream_t st);
}  // namespace batch

namespace {

using namespace stencil;
using batch::GridBarrier;
using batch::InstDev;

// Diagnostics: block (r, i) reduces rows r, r + B, ... of instance i.
template <typename T>
__global__ void __launch_bounds__(reduce::kThreads)
    batch_diag_partial(const InstDev<T> *__restrict__ inst, int first, int parity,
                       double *__restrict__ part)
{
    const int i = first + blockIdx.y;
    const InstDev<T> &I = inst[i];
    reduce::Acc a;
    if constexpr (sizeof(T) == 4)
        a = reduce::rows_f32<true, true>((const float *)I.b[parity], (const float *)I.n[parity],
                                         I.nx, I.ny, I.pitch, I.fth, blockIdx.x, gridDim.x);
    else
        a = reduce::rows_f64<true>((const double *)I.b[parity], (const double *)I.n[parity], I.nx,
                                   I.ny, I.pitch, I.bth, blockIdx.x, gridDim.x);
    a = reduce::block_reduce(a);
    if (threadIdx.x == 0)
        reduce::store_acc(part + 8LL * ((long long)i * gridDim.x + blockIdx.x), a);
}

__global__ void __launch_bounds__(reduce::kThreads)
    batch_diag_final(const double *__restrict__ part, int blocks, double *__restrict__ out)
{
    const int i = blockIdx.x;
    reduce::Acc a = reduce::empty_acc();
    for (int r = threadIdx.x; r < blocks; r += reduce::kThreads)
        reduce::combine(a, reduce::load_acc(part + 8LL * ((long long)i * blocks + r)));
    a = reduce::block_reduce(a);
    if (threadIdx.x == 0) reduce::store_acc(out + 8LL * i, a);
}

// (law, mobility) of a run -> the instantiation that serves it
#define CX_BATCH_DISPATCH(FN, ...)                                                          \
    (law == CX_CHEMO_RECEPTOR                                                               \
         ? (mob == CX_MOBILITY_CENTRAL                                                      \
                ? batch::FN<T, CX_CHEMO_RECEPTOR, CX_MOBILITY_CENTRAL>(__VA_ARGS__)          \
                : batch::FN<T, CX_CHEMO_RECEPTOR, CX_MOBILITY_UPWIND>(__VA_ARGS__))          \
         : (mob == CX_MOBILITY_CENTRAL                                                      \
                ? batch::FN<T, CX_CHEMO_CONSTANT, CX_MOBILITY_CENTRAL>(__VA_ARGS__)          \
                : batch::FN<T, CX_CHEMO_CONSTANT, CX_MOBILITY_UPWIND>(__VA_ARGS__)))

template <typename T>
cudaError_t launch_fused_prec(int law, int mob, const void *inst, const int4 *work, int nwork,
                              int parity, int rows, int heun, const BatchNoise &nz, cudaStream_t st)
{
    return CX_BATCH_DISPATCH(launch_fused_lm, inst, work, nwork, parity, rows, heun, nz.on,
                             nz.step_base, nz.step_off, st);
}

template <typename T>
cudaError_t launch_batch_prec(int law, int mob, const void *inst, const int4 *work, int nwork,
                              int parity, int rows, int stage, const BatchNoise &nz, cudaStream_t st)
{
    return CX_BATCH_DISPATCH(launch_step_lm, inst, work, nwork, parity, rows, stage, nz.on,
                             nz.step_base, nz.step_off, st);
}

template <typename T>
cudaError_t launch_resident_prec(int law, int mob, const void *inst, const int4 *work, int nwork,
                                 int parity, int rows, int nsteps, int heun, void *gb, long long spin,
                                 const BatchNoise &nz, cudaStream_t st)
{
    return CX_BATCH_DISPATCH(launch_resident_lm, inst, work, nwork, parity, rows, nsteps, heun,
                             nz.on, gb, spin, nz.step_base, nz.step_off, st);
}

#undef CX_BATCH_DISPATCH

// Writes the time step the next batch pass starts from (per-step noise).
__global__ void set_step_kernel(long long *p, long long v) { *p = v; }

}  // namespace

size_t grid_barrier_bytes() { return sizeof(GridBarrier); }

cudaError_t launch_batch_resident(int prec, int law, int mob, const void *inst, const int4 *work,
                                  int nwork, int parity, int rows, int nsteps, int heun,
                                  void *barrier, long long spin_limit, const BatchNoise &nz,
                                  cudaStream_t st)
{
    return prec == CX_PREC_F64
               ? launch_resident_prec<double>(law, mob, inst, work, nwork, parity, rows, nsteps, heun, barrier, spin_limit, nz, st)
               : launch_resident_prec<float>(law, mob, inst, work, nwork, parity, rows, nsteps, heun, barrier, spin_limit, nz, st);
}

cudaError_t launch_batch_step(int prec, int law, int mob, const void *inst, const int4 *work,
                              int nwork, int parity, int rows, int stage, const BatchNoise &nz,
                              cudaStream_t st)
{
    return prec == CX_PREC_F64
               ? launch_batch_prec<double>(law, mob, inst, work, nwork, parity, rows, stage, nz, st)
               : launch_batch_prec<float>(law, mob, inst, work, nwork, parity, rows, stage, nz, st);
}

cudaError_t launch_batch_fused(int prec, int law, int mob, const void *inst, const int4 *work,
                               int nwork, int parity, int rows, int heun, const BatchNoise &nz,
                               cudaStream_t st)
{
    return prec == CX_PREC_F64
               ? launch_fused_prec<double>(law, mob, inst, work, nwork, parity, rows, heun, nz, st)
               : launch_fused_prec<float>(law, mob, inst, work, nwork, parity, rows, heun, nz, st);
}

cudaError_t launch_set_step(long long *step_base, long long step, cudaStream_t st)
{
    set_step_kernel<<<1, 1, 0, st>>>(step_base, step);
    return cudaGetLastError();
}

cudaError_t launch_batch_diag(int prec, const void *inst, int first, int count, int blocks,
                              int parity, double *part, double *out, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    const dim3 g(blocks, count);
    if (prec == CX_PREC_F64)
        batch_diag_partial<double><<<g, reduce::kThreads, 0, st>>>((const InstDev<double> *)inst,
                                                                   first, parity, part);
    else
        batch_diag_partial<float><<<g, reduce::kThreads, 0, st>>>((const InstDev<float> *)inst,
                                                                  first, parity, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    batch_diag_final<<<count, reduce::kThreads, 0, st>>>(part + 8LL * first * blocks, blocks,
                                                         out + 8LL * first);
    return cudaGetLastError();
}

size_t inst_dev_bytes(int prec) { return prec == CX_PREC_F64 ? sizeof(InstDev<double>) : sizeof(InstDev<float>); }

// Host-side fill of one table entry (the table is copied to the device whole).
void fill_inst(int prec, void *table, int i, void *b0, void *b1, void *n0, void *n1, void *s,
               int nx, int ny, long long pitch, const Coef &k, double bth, uint64_t seed,
               double sigma0, double amp, int dist)
{
    if (prec == CX_PREC_F64) {
        InstDev<double> &d = ((InstDev<double> *)table)[i];
        d.b[0] = (double *)b0; d.b[1] = (double *)b1; d.n[0] = (double *)n0; d.n[1] = (double *)n1;
        d.s = (const double *)s;
        d.nx = nx; d.ny = ny; d.pitch = pitch;
        d.k = CoefT<double>{k.cA, k.cChi, k.cG, k.cR, k.cN};
        d.fth = reduce::float_threshold(bth);
        d.bth = bth;
        d.seed = seed;
        d.sigma0 = sigma0;
        d.amp = amp;
        d.dist = dist;
    } else {
        InstDev<float> &d = ((InstDev<float> *)table)[i];
        d.b[0] = (float *)b0; d.b[1] = (float *)b1; d.n[0] = (float *)n0; d.n[1] = (float *)n1;
        d.s = (const float *)s;
        d.nx = nx; d.ny = ny; d.pitch = pitch;
        d.k = CoefT<float>{(float)k.cA, (float)k.cChi, (float)k.cG, (float)k.cR, (float)k.cN};
        d.fth = reduce::float_threshold(bth);
        d.bth = bth;
        d.seed = seed;
        d.sigma0 = (float)sigma0;
        d.amp = (float)amp;
        d.dist = dist;
    }
}

}  // namespace cx
