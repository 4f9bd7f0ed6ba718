// cx_fused.cu -- one pass that takes two explicit stages of Eq. ka-chem-model
// (temporal blocking of depth 2; the march is in cx_fused.cuh).
//
//   HEUN 0  two forward-Euler steps, step and step + 1 (per-step noise draws
//           each step's sigma)
//   HEUN 1  one Heun step (second-order Runge-Kutta, Sec. 3): the first
//           stage u* = u + dt r(u) stays in registers and the pass writes
//           (u + u* + dt r(u*)) / 2; one sigma for both stages
//
// The pass reads the state (and the static sigma field) once and writes the
// state once: 20 B per cell per pass in FP32 with static noise, i.e. 10 B
// per Euler step instead of 20.  Input and output buffers differ (a tile's
// halo rows belong to its neighbours' input).
#include "cx_fused.cuh"

namespace cx {
namespace {

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

template <typename T, int LAW, int MOB, int NOISE, bool HEUN>
__global__ void __launch_bounds__(kThreads, fused_min_blocks<T>())
    fused_kernel(Ptrs<T> P, int nx, int ny, long long pitch, KV<P2<T>> k, NoiseT<T> nz1,
                 NoiseT<T> nz2, int rows)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int xb = blockIdx.x * kFusedBlockCols;  // first written column of the block
    // warps share nothing, so a warp whose written columns all lie past the
    // row's end (ragged last tile) leaves at once
    if (xb + warp * kFusedCols >= nx) return;
    const int x0 = xb + warp * kFusedCols - kCells + lane * kCells;
    const int j0 = blockIdx.y * rows;
    const int jend = min(j0 + rows, ny);
    // every column the block holds, xb - 4 .. xb + 483, lies inside the grid
    const bool interior = blockIdx.x > 0 && xb + kFusedBlockCols + kCells <= nx;
    if (blockIdx.y & 1) {
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
    NoiseT<T> nz2 = nz1;
    if (!HEUN) nz2.step = (uint64_t)a.step + 1;
    Ptrs<T> P{(const T *)a.b, (const T *)a.n, (const T *)a.s, nullptr, nullptr, (T *)a.bo,
              (T *)a.no};
    const dim3 grid((a.nx + kFusedBlockCols - 1) / kFusedBlockCols, (a.ny + a.rows - 1) / a.rows);
    fused_kernel<T, LAW, MOB, NOISE, HEUN><<<grid, kThreads, 0, st>>>(P, a.nx, a.ny, a.pitch, k,
                                                                      nz1, nz2, a.rows);
    return cudaGetLastError();
}

template <typename T, int LAW, int MOB>
cudaError_t launch_ns(const StepArgs &a, bool heun, cudaStream_t st)
{
    if (a.sg.per_step)
        return heun ? launch_t<T, LAW, MOB, 1, true>(a, st) : launch_t<T, LAW, MOB, 1, false>(a, st);
    return heun ? launch_t<T, LAW, MOB, 0, true>(a, st) : launch_t<T, LAW, MOB, 0, false>(a, st);
}

template <typename T>
cudaError_t launch_prec(const StepArgs &a, bool heun, cudaStream_t st)
{
    if (a.law == CX_CHEMO_RECEPTOR)
        return a.mob == CX_MOBILITY_CENTRAL
                   ? launch_ns<T, CX_CHEMO_RECEPTOR, CX_MOBILITY_CENTRAL>(a, heun, st)
                   : launch_ns<T, CX_CHEMO_RECEPTOR, CX_MOBILITY_UPWIND>(a, heun, st);
    return a.mob == CX_MOBILITY_CENTRAL
               ? launch_ns<T, CX_CHEMO_CONSTANT, CX_MOBILITY_CENTRAL>(a, heun, st)
               : launch_ns<T, CX_CHEMO_CONSTANT, CX_MOBILITY_UPWIND>(a, heun, st);
}

}  // namespace

cudaError_t launch_fused(int prec, const StepArgs &a, int heun, cudaStream_t st)
{
    return prec == CX_PREC_F64 ? launch_prec<double>(a, heun != 0, st)
                               : launch_prec<float>(a, heun != 0, st);
}

}  // namespace cx
