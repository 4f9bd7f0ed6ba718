// cx_fused_kernels.cuh -- the two-stage pass kernel (march in cx_fused.cuh)
// and its launch templates.  Included only by cx_fused_inst.cu, which the
// build compiles once per (precision, chemotaxis law, mobility) so that the
// sets of kernels compile in parallel; cx_fused.cu dispatches to them.
#pragma once

#include "cx_fused.cuh"

namespace cx {
namespace fused {

using namespace stencil;

// Resident blocks per SM the register budget is sized for: FP32 4 (at most
// 128 registers; with 96 the march's steady state spills, and 5 blocks per
// SM ran 6 % slower than 4), FP64 2 (bound by the FP64 pipe, not by
// occupancy).
#ifndef CX_FUSED_MIN_BLOCKS_F32
#define CX_FUSED_MIN_BLOCKS_F32 4
#endif
template <typename T> constexpr int fused_min_blocks()
{
    return sizeof(T) == 4 ? CX_FUSED_MIN_BLOCKS_F32 : 2;
}

template <typename T, int LAW, int MOB, int NOISE, bool HEUN, bool OFF32>
__global__ void __launch_bounds__(fused_threads<NOISE>(),
                                  fused_min_blocks<T>() * (kThreads / fused_threads<NOISE>()))
    fused_kernel(Ptrs<T> P, int nx, int ny, long long pitch, KV<P2<T>> k, NoiseT<T> nz1,
                 NoiseT<T> nz2, int rows)
{
    constexpr int kBlockCols = (fused_threads<NOISE>() / 32) * kFusedCols;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int xb = blockIdx.x * kBlockCols;  // first written column of the block
    // warps share nothing, so a warp whose written columns all lie past the
    // row's end (ragged last tile) leaves at once
    if (xb + warp * kFusedCols >= nx) return;
    const int x0 = xb + warp * kFusedCols - kCells + lane * kCells;
    const int j0 = blockIdx.y * rows;
    const int jend = min(j0 + rows, ny);
    // every column the block holds, xb - 4 .. xb + kBlockCols + 3, lies inside the grid
    const bool interior = blockIdx.x > 0 && xb + kBlockCols + kCells <= nx;
    if (blockIdx.y & 1) {
        if (interior)
            march2<T, LAW, MOB, NOISE, HEUN, -1, true, OFF32>(P, nx, ny, pitch, k, nz1, nz2, x0, j0,
                                                                 jend);
        else
            march2<T, LAW, MOB, NOISE, HEUN, -1, false, OFF32>(P, nx, ny, pitch, k, nz1, nz2, x0, j0,
                                                                 jend);
    } else {
        if (interior)
            march2<T, LAW, MOB, NOISE, HEUN, +1, true, OFF32>(P, nx, ny, pitch, k, nz1, nz2, x0, j0,
                                                                 jend);
        else
            march2<T, LAW, MOB, NOISE, HEUN, +1, false, OFF32>(P, nx, ny, pitch, k, nz1, nz2, x0, j0,
                                                                 jend);
    }
}

template <typename T, int LAW, int MOB, int NOISE, bool HEUN>
cudaError_t launch_t(const StepArgs &a, cudaStream_t st)
{
    const KV<P2<T>> k = make_kv(CoefT<T>{(T)a.k.cA, (T)a.k.cChi, (T)a.k.cG, (T)a.k.cR, (T)a.k.cN});
    NoiseT<T> nz1;
    nz1.seed = a.sg.seed;
    nz1.step = (uint64_t)a.step;
    nz1.dist = a.sg.dist;
    nz1.sigma0 = (T)a.sg.sigma0;
    nz1.amp = (T)a.sg.amp;
    set_noise_keys(nz1);
    NoiseT<T> nz2 = nz1;
    if (!HEUN) nz2.step = (uint64_t)a.step + 1;
    Ptrs<T> P{(const T *)a.b, (const T *)a.n, (const T *)a.s, nullptr, nullptr, (T *)a.bo,
              (T *)a.no};
    constexpr int threads = fused_threads<NOISE>();
    constexpr int cols = (threads / 32) * kFusedCols;
    const dim3 grid((a.nx + cols - 1) / cols, (a.ny + a.rows - 1) / a.rows);
    // 32-bit element offsets for the per-step passes when every offset fits
    if (NOISE == 1 && (long long)a.ny * a.pitch < (1LL << 31))
        fused_kernel<T, LAW, MOB, NOISE, HEUN, NOISE == 1><<<grid, threads, 0, st>>>(
            P, a.nx, a.ny, a.pitch, k, nz1, nz2, a.rows);
    else
        fused_kernel<T, LAW, MOB, NOISE, HEUN, false><<<grid, threads, 0, st>>>(
            P, a.nx, a.ny, a.pitch, k, nz1, nz2, a.rows);
    return cudaGetLastError();
}

// One (precision, law, mobility) combination: every noise mode and scheme.
template <typename T, int LAW, int MOB>
cudaError_t launch_fused_lm(const StepArgs &a, bool heun, cudaStream_t st)
{
    if (a.sg.per_step)
        return heun ? launch_t<T, LAW, MOB, 1, true>(a, st) : launch_t<T, LAW, MOB, 1, false>(a, st);
    return heun ? launch_t<T, LAW, MOB, 0, true>(a, st) : launch_t<T, LAW, MOB, 0, false>(a, st);
}

}  // namespace fused
}  // namespace cx
