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
// Every instance goes through the same per-thread stencil code as a single
// grid (cx_stencil.cuh), so a batch instance and a cx_ctx with the same
// grid, parameters and seed give bit-identical fields.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "cx_reduce.cuh"
#include "cx_stencil.cuh"

namespace cx {
namespace {

using namespace stencil;

template <typename T> struct InstDev {
    T *b[2];
    T *n[2];
    const T *s;
    int nx, ny;
    long long pitch;
    CoefT<T> k;
    float fth;     // FP32 envelope threshold (diagnostics)
    double bth;    // FP64 envelope threshold
};

// stage 0: u_out(parity^1) = u(parity) + dt r(u(parity))
// stage 1: u(parity) = (u(parity) + u*(parity^1) + dt r(u*)) / 2, in place
template <typename T, int LAW, int MOB, int STAGE>
__global__ void __launch_bounds__(kThreads)
    batch_step_kernel(const InstDev<T> *__restrict__ inst, const int4 *__restrict__ work,
                      int parity, int rows)
{
    const int4 w = work[blockIdx.x];
    const InstDev<T> &I = inst[w.x];
    const int nx = I.nx, ny = I.ny;
    const long long pitch = I.pitch;
    const CoefT<T> k = I.k;
    Ptrs<T> P;
    if (STAGE == 0) {
        P = Ptrs<T>{I.b[parity], I.n[parity], I.s, nullptr, nullptr, I.b[parity ^ 1],
                    I.n[parity ^ 1]};
    } else {
        P = Ptrs<T>{I.b[parity ^ 1], I.n[parity ^ 1], I.s, I.b[parity], I.n[parity],
                    I.b[parity], I.n[parity]};
    }
    NoiseT<T> nz{};
    const int x0 = (w.y * kThreads + threadIdx.x) * kCells;
    const int j0 = w.z * rows;
    const int jend = min(j0 + rows, ny);
    if (w.z & 1)
        march<T, LAW, MOB, 0, STAGE, -1>(P, nx, ny, pitch, k, nz, x0, j0, jend);
    else
        march<T, LAW, MOB, 0, STAGE, +1>(P, nx, ny, pitch, k, nz, x0, j0, jend);
}

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
        a = reduce::rows_f32<true>((const float *)I.b[parity], (const float *)I.n[parity], I.nx,
                                   I.ny, I.pitch, I.fth, blockIdx.x, gridDim.x);
    else
        a = reduce::rows_f64((const double *)I.b[parity], (const double *)I.n[parity], I.nx, I.ny,
                             I.pitch, I.bth, blockIdx.x, gridDim.x);
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

template <typename T, int LAW, int MOB>
cudaError_t launch_batch_t(const void *inst, const int4 *work, int nwork, int parity, int rows,
                           int stage, cudaStream_t st)
{
    if (nwork <= 0) return cudaSuccess;
    if (stage == 0)
        batch_step_kernel<T, LAW, MOB, 0><<<nwork, kThreads, 0, st>>>((const InstDev<T> *)inst, work,
                                                                      parity, rows);
    else
        batch_step_kernel<T, LAW, MOB, 1><<<nwork, kThreads, 0, st>>>((const InstDev<T> *)inst, work,
                                                                      parity, rows);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_batch_prec(int law, int mob, const void *inst, const int4 *work, int nwork,
                              int parity, int rows, int stage, cudaStream_t st)
{
    if (law == CX_CHEMO_RECEPTOR)
        return mob == CX_MOBILITY_CENTRAL
                   ? launch_batch_t<T, CX_CHEMO_RECEPTOR, CX_MOBILITY_CENTRAL>(inst, work, nwork, parity, rows, stage, st)
                   : launch_batch_t<T, CX_CHEMO_RECEPTOR, CX_MOBILITY_UPWIND>(inst, work, nwork, parity, rows, stage, st);
    return mob == CX_MOBILITY_CENTRAL
               ? launch_batch_t<T, CX_CHEMO_CONSTANT, CX_MOBILITY_CENTRAL>(inst, work, nwork, parity, rows, stage, st)
               : launch_batch_t<T, CX_CHEMO_CONSTANT, CX_MOBILITY_UPWIND>(inst, work, nwork, parity, rows, stage, st);
}

}  // namespace

cudaError_t launch_batch_step(int prec, int law, int mob, const void *inst, const int4 *work,
                              int nwork, int parity, int rows, int stage, cudaStream_t st)
{
    return prec == CX_PREC_F64
               ? launch_batch_prec<double>(law, mob, inst, work, nwork, parity, rows, stage, st)
               : launch_batch_prec<float>(law, mob, inst, work, nwork, parity, rows, stage, st);
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
               int nx, int ny, long long pitch, const Coef &k, double bth)
{
    if (prec == CX_PREC_F64) {
        InstDev<double> &d = ((InstDev<double> *)table)[i];
        d.b[0] = (double *)b0; d.b[1] = (double *)b1; d.n[0] = (double *)n0; d.n[1] = (double *)n1;
        d.s = (const double *)s;
        d.nx = nx; d.ny = ny; d.pitch = pitch;
        d.k = CoefT<double>{k.cA, k.cChi, k.cG, k.cR, k.cN};
        d.fth = reduce::float_threshold(bth);
        d.bth = bth;
    } else {
        InstDev<float> &d = ((InstDev<float> *)table)[i];
        d.b[0] = (float *)b0; d.b[1] = (float *)b1; d.n[0] = (float *)n0; d.n[1] = (float *)n1;
        d.s = (const float *)s;
        d.nx = nx; d.ny = ny; d.pitch = pitch;
        d.k = CoefT<float>{(float)k.cA, (float)k.cChi, (float)k.cG, (float)k.cR, (float)k.cN};
        d.fth = reduce::float_threshold(bth);
        d.bth = bth;
    }
}

}  // namespace cx
