// cx_batch_kernels.cuh -- the batch step kernels (one and two stages per
// pass, and the resident cooperative form) and their launch templates.
// Included only by cx_batch_inst.cu, which the build compiles once per
// (precision, chemotaxis law, mobility) so that the sets of kernels compile
// in parallel; cx_batch.cu dispatches to them.
#pragma once

#include "cx_batch_types.cuh"
#include "cx_fused.cuh"

namespace cx {
namespace batch {

using namespace stencil;

// One tile (work item w) of one step.
// stage 0: u_out(parity^1) = u(parity) + dt r(u(parity))
// stage 1: u(parity) = (u(parity) + u*(parity^1) + dt r(u*)) / 2, in place
// NOISE 1: sigma is redrawn for time step `step` (both Heun stages share it).
template <typename T, int LAW, int MOB, int NOISE, int STAGE, bool CG>
__device__ __forceinline__ void tile_step(const InstDev<T> *__restrict__ inst, const int4 w,
                                          int parity, int rows, uint64_t step)
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
    const NoiseT<T> nz = NOISE ? inst_noise(I, step) : NoiseT<T>{};
    const int x0 = (w.y * kThreads + threadIdx.x) * kCells;
    const int j0 = w.z * rows;
    const int jend = min(j0 + rows, ny);
    const bool interior = w.y > 0 && (w.y + 1) * kThreads * kCells < nx;
    if (w.z & 1) {
        if (interior)
            march<T, LAW, MOB, NOISE, STAGE, -1, CG, true>(P, nx, ny, pitch, k, nz, x0, j0, jend);
        else
            march<T, LAW, MOB, NOISE, STAGE, -1, CG>(P, nx, ny, pitch, k, nz, x0, j0, jend);
    } else {
        if (interior)
            march<T, LAW, MOB, NOISE, STAGE, +1, CG, true>(P, nx, ny, pitch, k, nz, x0, j0, jend);
        else
            march<T, LAW, MOB, NOISE, STAGE, +1, CG>(P, nx, ny, pitch, k, nz, x0, j0, jend);
    }
}

// Grid-wide barrier of a cooperative launch (every block is resident).  The
// wait is bounded: after spin_limit polls the block records a failure and
// leaves; a block that sees a recorded failure does not wait at all.
// Returns false (in every thread of the block) on failure.
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

// The time step of the first pass of a launch is *step_base + step_off:
// the host writes step_base before a captured graph is replayed, and the
// passes inside the graph add their fixed offsets (read only with NOISE 1).
template <typename T, int LAW, int MOB, int NOISE, int HEUN>
__global__ void __launch_bounds__(kThreads, resident_min_blocks<T>())
    batch_resident_kernel(const InstDev<T> *__restrict__ inst, const int4 *__restrict__ work,
                          int nwork, int parity, int rows, int nsteps, GridBarrier *gb,
                          long long spin_limit, const long long *__restrict__ step_base,
                          int step_off)
{
    const uint64_t step0 = NOISE ? (uint64_t)(__ldg(step_base) + step_off) : 0;
    for (int s = 0; s < nsteps; ++s) {
        for (int w = blockIdx.x; w < nwork; w += gridDim.x)
            tile_step<T, LAW, MOB, NOISE, 0, true>(inst, work[w], parity, rows, step0 + s);
        if (!grid_barrier(gb, spin_limit)) return;
        if (HEUN) {
            for (int w = blockIdx.x; w < nwork; w += gridDim.x)
                tile_step<T, LAW, MOB, NOISE, 1, true>(inst, work[w], parity, rows, step0 + s);
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

template <typename T, int LAW, int MOB, int NOISE, int STAGE>
__global__ void __launch_bounds__(kThreads, batch_min_blocks<T, STAGE>())
    batch_step_kernel(const InstDev<T> *__restrict__ inst, const int4 *__restrict__ work,
                      int parity, int rows, const long long *__restrict__ step_base, int step_off)
{
    const uint64_t step = NOISE ? (uint64_t)(__ldg(step_base) + step_off) : 0;
    tile_step<T, LAW, MOB, NOISE, STAGE, false>(inst, work[blockIdx.x], parity, rows, step);
}

// Two stages per pass (two Euler steps, or one Heun step) of one tile of the
// 120-column work list, one warp per block: reads u(parity), writes
// u(parity^1).  One-warp blocks fit the sweep's 512..2048-wide instances,
// which four-warp (480-column) tiles cover with partly idle blocks.
// Register budget as the single-grid two-stage pass (128 registers in FP32).
constexpr int kBatchFusedThreads = 32;
template <typename T> constexpr int batch_fused_min_blocks() { return sizeof(T) == 4 ? 16 : 8; }

template <typename T, int LAW, int MOB, int NOISE, bool HEUN>
__global__ void __launch_bounds__(kBatchFusedThreads, batch_fused_min_blocks<T>())
    batch_fused_kernel(const InstDev<T> *__restrict__ inst, const int4 *__restrict__ work,
                       int parity, int rows, const long long *__restrict__ step_base, int step_off)
{
    const int4 w = work[blockIdx.x];
    const InstDev<T> &I = inst[w.x];
    const int nx = I.nx, ny = I.ny;
    const long long pitch = I.pitch;
    const KV<P2<T>> k = make_kv(I.k);
    const Ptrs<T> P{I.b[parity], I.n[parity], I.s, nullptr, nullptr, I.b[parity ^ 1],
                    I.n[parity ^ 1]};
    // NOISE 1: stage one draws sigma for the pass's first step; Euler's
    // second stage for the next step, Heun's second stage shares the first's
    const uint64_t step = NOISE ? (uint64_t)(__ldg(step_base) + step_off) : 0;
    const NoiseT<T> nz1 = NOISE ? inst_noise(I, step) : NoiseT<T>{};
    const NoiseT<T> nz2 = NOISE && !HEUN ? inst_noise(I, step + 1) : nz1;
    const int lane = threadIdx.x & 31;
    const int xb = w.y * kFusedCols;  // first written column of the tile
    const int x0 = xb - kCells + lane * kCells;
    const int j0 = w.z * rows;
    const int jend = min(j0 + rows, ny);
    // every column the warp holds, xb - 4 .. xb + 123, lies inside the grid
    const bool interior = w.y > 0 && xb + kFusedCols + kCells <= nx;
    if (w.z & 1) {
        if (interior)
            march2<T, LAW, MOB, NOISE, HEUN, -1, true>(P, nx, ny, pitch, k, nz1, nz2, x0, j0, jend);
        else
            march2<T, LAW, MOB, NOISE, HEUN, -1, false>(P, nx, ny, pitch, k, nz1, nz2, x0, j0, jend);
    } else {
        if (interior)
            march2<T, LAW, MOB, NOISE, HEUN, +1, true>(P, nx, ny, pitch, k, nz1, nz2, x0, j0, jend);
        else
            march2<T, LAW, MOB, NOISE, HEUN, +1, false>(P, nx, ny, pitch, k, nz1, nz2, x0, j0, jend);
    }
}

template <typename T, int LAW, int MOB, int NOISE>
cudaError_t launch_step_n(const void *inst, const int4 *work, int nwork, int parity, int rows,
                          int stage, const long long *step_base, int step_off, cudaStream_t st)
{
    const InstDev<T> *ip = (const InstDev<T> *)inst;
    if (stage == 0)
        batch_step_kernel<T, LAW, MOB, NOISE, 0><<<nwork, kThreads, 0, st>>>(ip, work, parity, rows,
                                                                             step_base, step_off);
    else
        batch_step_kernel<T, LAW, MOB, NOISE, 1><<<nwork, kThreads, 0, st>>>(ip, work, parity, rows,
                                                                             step_base, step_off);
    return cudaGetLastError();
}

template <typename T, int LAW, int MOB>
cudaError_t launch_step_lm(const void *inst, const int4 *work, int nwork, int parity, int rows,
                           int stage, int noise, const long long *step_base, int step_off,
                           cudaStream_t st)
{
    if (nwork <= 0) return cudaSuccess;
    return noise ? launch_step_n<T, LAW, MOB, 1>(inst, work, nwork, parity, rows, stage, step_base, step_off, st)
                 : launch_step_n<T, LAW, MOB, 0>(inst, work, nwork, parity, rows, stage, step_base, step_off, st);
}

template <typename T, int LAW, int MOB, int NOISE>
cudaError_t launch_fused_n(const void *inst, const int4 *work, int nwork, int parity, int rows,
                           int heun, const long long *step_base, int step_off, cudaStream_t st)
{
    const InstDev<T> *ip = (const InstDev<T> *)inst;
    if (heun)
        batch_fused_kernel<T, LAW, MOB, NOISE, true><<<nwork, kBatchFusedThreads, 0, st>>>(
            ip, work, parity, rows, step_base, step_off);
    else
        batch_fused_kernel<T, LAW, MOB, NOISE, false><<<nwork, kBatchFusedThreads, 0, st>>>(
            ip, work, parity, rows, step_base, step_off);
    return cudaGetLastError();
}

template <typename T, int LAW, int MOB>
cudaError_t launch_fused_lm(const void *inst, const int4 *work, int nwork, int parity, int rows,
                            int heun, int noise, const long long *step_base, int step_off,
                            cudaStream_t st)
{
    if (nwork <= 0) return cudaSuccess;
    return noise ? launch_fused_n<T, LAW, MOB, 1>(inst, work, nwork, parity, rows, heun, step_base, step_off, st)
                 : launch_fused_n<T, LAW, MOB, 0>(inst, work, nwork, parity, rows, heun, step_base, step_off, st);
}

// Cooperative launch of the resident kernel with as many blocks as can be
// resident at once (at most one per tile), so every block reaches every
// barrier.
template <typename T, int LAW, int MOB, int NOISE, int HEUN>
cudaError_t launch_resident_h(const void *inst, const int4 *work, int nwork, int parity, int rows,
                              int nsteps, void *gb, long long spin, const long long *step_base,
                              int step_off, cudaStream_t st)
{
    if (nwork <= 0 || nsteps <= 0) return cudaSuccess;
    const void *kern = (const void *)batch_resident_kernel<T, LAW, MOB, NOISE, HEUN>;
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, batch_resident_kernel<T, LAW, MOB, NOISE, HEUN>, kThreads, 0);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    int grid = per_sm * sms;
    if (grid > nwork) grid = nwork;
    if (grid < 1) return cudaErrorCooperativeLaunchTooLarge;
    const InstDev<T> *ip = (const InstDev<T> *)inst;
    GridBarrier *gp = (GridBarrier *)gb;
    void *args[] = {(void *)&ip, (void *)&work, (void *)&nwork, (void *)&parity, (void *)&rows,
                    (void *)&nsteps, (void *)&gp, (void *)&spin, (void *)&step_base,
                    (void *)&step_off};
    return cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(kThreads), args, 0, st);
}

template <typename T, int LAW, int MOB>
cudaError_t launch_resident_lm(const void *inst, const int4 *work, int nwork, int parity, int rows,
                               int nsteps, int heun, int noise, void *gb, long long spin,
                               const long long *step_base, int step_off, cudaStream_t st)
{
    if (noise)
        return heun ? launch_resident_h<T, LAW, MOB, 1, 1>(inst, work, nwork, parity, rows, nsteps, gb, spin, step_base, step_off, st)
                    : launch_resident_h<T, LAW, MOB, 1, 0>(inst, work, nwork, parity, rows, nsteps, gb, spin, step_base, step_off, st);
    return heun ? launch_resident_h<T, LAW, MOB, 0, 1>(inst, work, nwork, parity, rows, nsteps, gb, spin, step_base, step_off, st)
                : launch_resident_h<T, LAW, MOB, 0, 0>(inst, work, nwork, parity, rows, nsteps, gb, spin, step_base, step_off, st);
}

}  // namespace batch
}  // namespace cx
