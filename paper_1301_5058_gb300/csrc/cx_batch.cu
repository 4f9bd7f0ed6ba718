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
// one entry per 480-column x `rows`-row tile of the two-stage march.
//
// Every instance goes through the same per-thread stencil code as a single
// grid (cx_stencil.cuh, cx_fused.cuh), so a batch instance and a cx_ctx with
// the same grid, parameters and seed give bit-identical fields.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "cx_fused.cuh"
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

// One tile (work item w) of one step.
// stage 0: u_out(parity^1) = u(parity) + dt r(u(parity))
// stage 1: u(parity) = (u(parity) + u*(parity^1) + dt r(u*)) / 2, in place
template <typename T, int LAW, int MOB, int STAGE, bool CG>
__device__ __forceinline__ void tile_step(const InstDev<T> *__restrict__ inst, const int4 w,
                                          int parity, int rows)
{
    const InstDev<T> &I = inst[w.x];
    const int nx = I.nx, ny = I.ny;
    const long long pitch = I.pitch;
    const KV<P2<T>> k = make_kv(I.k);
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
    const bool interior = w.y > 0 && (w.y + 1) * kThreads * kCells < nx;
    if (w.z & 1) {
        if (interior)
            march<T, LAW, MOB, 0, STAGE, -1, CG, true>(P, nx, ny, pitch, k, nz, x0, j0, jend);
        else
            march<T, LAW, MOB, 0, STAGE, -1, CG>(P, nx, ny, pitch, k, nz, x0, j0, jend);
    } else {
        if (interior)
            march<T, LAW, MOB, 0, STAGE, +1, CG, true>(P, nx, ny, pitch, k, nz, x0, j0, jend);
        else
            march<T, LAW, MOB, 0, STAGE, +1, CG>(P, nx, ny, pitch, k, nz, x0, j0, jend);
    }
}

// Grid-wide barrier of a cooperative launch (every block is resident).  The
// wait is bounded: after spin_limit polls the block records a failure and
// leaves; a block that sees a recorded failure does not wait at all.
// Returns false (in every thread of the block) on failure.
struct GridBarrier {
    unsigned count, gen;
    int err, pad;
};

__device__ __forceinline__ bool grid_barrier(GridBarrier *gb, long long spin_limit)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile GridBarrier *v = gb;
        ok = v->err ? 0 : 1;
        if (ok) {
            const unsigned g = v->gen;
            __threadfence();  // this block's writes before its arrival
            const unsigned arrived = atomicAdd(&gb->count, 1u) + 1u;
            if (arrived == gridDim.x) {
                atomicExch(&gb->count, 0u);
                __threadfence();
                atomicAdd(&gb->gen, 1u);
            } else {
                long long it = 0;
                while (v->gen == g) {
                    if (++it > spin_limit) {
                        atomicExch(&gb->err, 1);
                        ok = 0;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __threadfence();  // the other blocks' writes before this block reads
            if (v->err) ok = 0;
        }
    }
    __syncthreads();
    return ok != 0;
}

// Several steps of a group of instances in one cooperative launch: the
// group's tiles are dealt to the resident blocks, and a grid barrier
// separates the steps (and Heun's stages).  Loads go through L2 only.
// Register budget: 2 blocks per SM (the launch sizes its grid from the
// occupancy this leaves).  The kernel inlines every march variant; its FP64
// Heun forms still spill a little at 255 registers.
template <typename T> constexpr int resident_min_blocks() { return 2; }

template <typename T, int LAW, int MOB, int HEUN>
__global__ void __launch_bounds__(kThreads, resident_min_blocks<T>())
    batch_resident_kernel(const InstDev<T> *__restrict__ inst, const int4 *__restrict__ work,
                          int nwork, int parity, int rows, int nsteps, GridBarrier *gb,
                          long long spin_limit)
{
    for (int s = 0; s < nsteps; ++s) {
        for (int w = blockIdx.x; w < nwork; w += gridDim.x)
            tile_step<T, LAW, MOB, 0, true>(inst, work[w], parity, rows);
        if (!grid_barrier(gb, spin_limit)) return;
        if (HEUN) {
            for (int w = blockIdx.x; w < nwork; w += gridDim.x)
                tile_step<T, LAW, MOB, 1, true>(inst, work[w], parity, rows);
            if (!grid_barrier(gb, spin_limit)) return;
        } else {
            parity ^= 1;
        }
    }
}

// stage 0: u_out(parity^1) = u(parity) + dt r(u(parity))
// stage 1: u(parity) = (u(parity) + u*(parity^1) + dt r(u*)) / 2, in place
// As the single-grid step kernel: FP32 Euler steps are bound by HBM
// bandwidth (64 registers, 8 blocks per SM); Heun's second stage 4; FP64 2.
template <typename T, int STAGE> constexpr int batch_min_blocks()
{
    return sizeof(T) == 4 ? (STAGE == 0 ? 8 : 4) : 2;
}

template <typename T, int LAW, int MOB, int STAGE>
__global__ void __launch_bounds__(kThreads, batch_min_blocks<T, STAGE>())
    batch_step_kernel(const InstDev<T> *__restrict__ inst, const int4 *__restrict__ work,
                      int parity, int rows)
{
    tile_step<T, LAW, MOB, STAGE, false>(inst, work[blockIdx.x], parity, rows);
}

// Two stages per pass (two Euler steps, or one Heun step) of one tile of the
// 480-column work list: reads u(parity), writes u(parity^1).  Register
// budget as the single-grid two-stage pass (128 registers in FP32).
template <typename T> constexpr int batch_fused_min_blocks() { return sizeof(T) == 4 ? 4 : 2; }

template <typename T, int LAW, int MOB, bool HEUN>
__global__ void __launch_bounds__(kThreads, batch_fused_min_blocks<T>())
    batch_fused_kernel(const InstDev<T> *__restrict__ inst, const int4 *__restrict__ work,
                       int parity, int rows)
{
    const int4 w = work[blockIdx.x];
    const InstDev<T> &I = inst[w.x];
    const int nx = I.nx, ny = I.ny;
    const long long pitch = I.pitch;
    const KV<P2<T>> k = make_kv(I.k);
    const Ptrs<T> P{I.b[parity], I.n[parity], I.s, nullptr, nullptr, I.b[parity ^ 1],
                    I.n[parity ^ 1]};
    const NoiseT<T> nz{};
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int xb = w.y * kFusedBlockCols;
    // warps share nothing: one whose written columns all lie past the row's
    // end (ragged last tile) leaves at once
    if (xb + warp * kFusedCols >= nx) return;
    const int x0 = xb + warp * kFusedCols - kCells + lane * kCells;
    const int j0 = w.z * rows;
    const int jend = min(j0 + rows, ny);
    const bool interior = w.y > 0 && xb + kFusedBlockCols + kCells <= nx;
    if (w.z & 1) {
        if (interior)
            march2<T, LAW, MOB, 0, HEUN, -1, true>(P, nx, ny, pitch, k, nz, nz, x0, j0, jend);
        else
            march2<T, LAW, MOB, 0, HEUN, -1, false>(P, nx, ny, pitch, k, nz, nz, x0, j0, jend);
    } else {
        if (interior)
            march2<T, LAW, MOB, 0, HEUN, +1, true>(P, nx, ny, pitch, k, nz, nz, x0, j0, jend);
        else
            march2<T, LAW, MOB, 0, HEUN, +1, false>(P, nx, ny, pitch, k, nz, nz, x0, j0, jend);
    }
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

template <typename T, int LAW, int MOB>
cudaError_t launch_fused_t(const void *inst, const int4 *work, int nwork, int parity, int rows,
                           int heun, cudaStream_t st)
{
    if (nwork <= 0) return cudaSuccess;
    if (heun)
        batch_fused_kernel<T, LAW, MOB, true><<<nwork, kThreads, 0, st>>>((const InstDev<T> *)inst,
                                                                          work, parity, rows);
    else
        batch_fused_kernel<T, LAW, MOB, false><<<nwork, kThreads, 0, st>>>((const InstDev<T> *)inst,
                                                                           work, parity, rows);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fused_prec(int law, int mob, const void *inst, const int4 *work, int nwork,
                              int parity, int rows, int heun, cudaStream_t st)
{
    if (law == CX_CHEMO_RECEPTOR)
        return mob == CX_MOBILITY_CENTRAL
                   ? launch_fused_t<T, CX_CHEMO_RECEPTOR, CX_MOBILITY_CENTRAL>(inst, work, nwork, parity, rows, heun, st)
                   : launch_fused_t<T, CX_CHEMO_RECEPTOR, CX_MOBILITY_UPWIND>(inst, work, nwork, parity, rows, heun, st);
    return mob == CX_MOBILITY_CENTRAL
               ? launch_fused_t<T, CX_CHEMO_CONSTANT, CX_MOBILITY_CENTRAL>(inst, work, nwork, parity, rows, heun, st)
               : launch_fused_t<T, CX_CHEMO_CONSTANT, CX_MOBILITY_UPWIND>(inst, work, nwork, parity, rows, heun, st);
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

// Cooperative launch of the resident kernel with as many blocks as can be
// resident at once (at most one per tile), so every block reaches every
// barrier.
template <typename T, int LAW, int MOB, int HEUN>
cudaError_t launch_resident_h(const void *inst, const int4 *work, int nwork, int parity, int rows,
                              int nsteps, void *gb, long long spin, cudaStream_t st)
{
    if (nwork <= 0 || nsteps <= 0) return cudaSuccess;
    const void *kern = (const void *)batch_resident_kernel<T, LAW, MOB, HEUN>;
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, batch_resident_kernel<T, LAW, MOB, HEUN>, kThreads, 0);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    int grid = per_sm * sms;
    if (grid > nwork) grid = nwork;
    if (grid < 1) return cudaErrorCooperativeLaunchTooLarge;
    const InstDev<T> *ip = (const InstDev<T> *)inst;
    GridBarrier *gp = (GridBarrier *)gb;
    void *args[] = {(void *)&ip, (void *)&work, (void *)&nwork, (void *)&parity, (void *)&rows,
                    (void *)&nsteps, (void *)&gp, (void *)&spin};
    return cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(kThreads), args, 0, st);
}

template <typename T, int LAW, int MOB>
cudaError_t launch_resident_t(const void *inst, const int4 *work, int nwork, int parity, int rows,
                              int nsteps, int heun, void *gb, long long spin, cudaStream_t st)
{
    return heun ? launch_resident_h<T, LAW, MOB, 1>(inst, work, nwork, parity, rows, nsteps, gb, spin, st)
                : launch_resident_h<T, LAW, MOB, 0>(inst, work, nwork, parity, rows, nsteps, gb, spin, st);
}

template <typename T>
cudaError_t launch_resident_prec(int law, int mob, const void *inst, const int4 *work, int nwork,
                                 int parity, int rows, int nsteps, int heun, void *gb, long long spin,
                                 cudaStream_t st)
{
    if (law == CX_CHEMO_RECEPTOR)
        return mob == CX_MOBILITY_CENTRAL
                   ? launch_resident_t<T, CX_CHEMO_RECEPTOR, CX_MOBILITY_CENTRAL>(inst, work, nwork, parity, rows, nsteps, heun, gb, spin, st)
                   : launch_resident_t<T, CX_CHEMO_RECEPTOR, CX_MOBILITY_UPWIND>(inst, work, nwork, parity, rows, nsteps, heun, gb, spin, st);
    return mob == CX_MOBILITY_CENTRAL
               ? launch_resident_t<T, CX_CHEMO_CONSTANT, CX_MOBILITY_CENTRAL>(inst, work, nwork, parity, rows, nsteps, heun, gb, spin, st)
               : launch_resident_t<T, CX_CHEMO_CONSTANT, CX_MOBILITY_UPWIND>(inst, work, nwork, parity, rows, nsteps, heun, gb, spin, st);
}

}  // namespace

size_t grid_barrier_bytes() { return sizeof(GridBarrier); }

cudaError_t launch_batch_resident(int prec, int law, int mob, const void *inst, const int4 *work,
                                  int nwork, int parity, int rows, int nsteps, int heun,
                                  void *barrier, long long spin_limit, cudaStream_t st)
{
    return prec == CX_PREC_F64
               ? launch_resident_prec<double>(law, mob, inst, work, nwork, parity, rows, nsteps, heun, barrier, spin_limit, st)
               : launch_resident_prec<float>(law, mob, inst, work, nwork, parity, rows, nsteps, heun, barrier, spin_limit, st);
}

cudaError_t launch_batch_step(int prec, int law, int mob, const void *inst, const int4 *work,
                              int nwork, int parity, int rows, int stage, cudaStream_t st)
{
    return prec == CX_PREC_F64
               ? launch_batch_prec<double>(law, mob, inst, work, nwork, parity, rows, stage, st)
               : launch_batch_prec<float>(law, mob, inst, work, nwork, parity, rows, stage, st);
}

cudaError_t launch_batch_fused(int prec, int law, int mob, const void *inst, const int4 *work,
                               int nwork, int parity, int rows, int heun, cudaStream_t st)
{
    return prec == CX_PREC_F64
               ? launch_fused_prec<double>(law, mob, inst, work, nwork, parity, rows, heun, st)
               : launch_fused_prec<float>(law, mob, inst, work, nwork, parity, rows, heun, st);
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
