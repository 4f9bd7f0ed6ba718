// cx_step.cu -- one fused explicit step of the bacteria/nutrient system
// (Eq. ka-chem-model in the general form of Eq. ka-model-dim, chemotactic
// flux of Eq. chemflux, no-flux walls of Eq. bconds).
//
// One pass per forward-Euler step reads b, n, sigma and writes b', n'
// (20 B per cell in FP32, 40 B in FP64).  Each thread owns 4 adjacent cells
// of a row (one 16-byte vector per FP32 field) and marches down one tile of
// `rows` rows (32 by default; a tuning knob),
// keeping the row ahead in registers, so every cell is loaded from HBM once
// and every y-face flux is evaluated once and reused by the two cells that
// share it.  x-neighbours come from the adjacent lanes by warp shuffles;
// lanes 0 and 31 fetch the one cell beyond the warp.  Boundary faces carry
// zero flux.
//
// Template switches:
//   NOISE 0  sigma read from its array (static field)
//   NOISE 1  sigma regenerated in registers from Philox for the time step
//            being taken (Sec. 3: redrawn at every grid point and step), so
//            the pass reads only b and n (16 B per FP32 cell)
//   STAGE 0  u_out = u + dt r(u): forward Euler, or Heun's first stage
//   STAGE 1  Heun's second stage u_out = (u0 + u* + dt r(u*)) / 2, reading
//            u0 pointwise and overwriting it in place (second-order
//            Runge-Kutta, Sec. 3)
#include "cx_stencil.cuh"

namespace cx {
namespace {

using namespace stencil;

// Row-bands alternate their march direction, so a halo row shared by two
// neighbouring bands is read by both near the start (or both near the end)
// of their marches, while it is still in L2, instead of once at the start
// of one band and again at the end of the other.
// Resident blocks per SM the register budget is sized for.  FP32 Euler with
// a static sigma field is bound by HBM bandwidth and needs every warp it can
// get: 64 registers, 8 blocks (32 warps).  Other FP32 forms: 4 (128
// registers); FP64 (bound by the FP64 pipe): 2.
template <typename T, int NOISE, int STAGE> constexpr int step_min_blocks()
{
    return sizeof(T) == 4 ? ((NOISE == 0 && STAGE == 0) ? 8 : 4) : 2;
}

template <typename T, int LAW, int MOB, int NOISE, int STAGE>
__global__ void __launch_bounds__(kThreads, step_min_blocks<T, NOISE, STAGE>())
    step_kernel(Ptrs<T> P, int nx, int ny, long long pitch, KV<P2<T>> k, NoiseT<T> nz, int rows)
{
    const int x0 = (blockIdx.x * kThreads + threadIdx.x) * kCells;
    const int j0 = blockIdx.y * rows;
    const int jend = min(j0 + rows, ny);
    // a block whose 512 columns touch neither x-wall takes the branch-free path
    const bool interior = blockIdx.x > 0 && (blockIdx.x + 1) * kThreads * kCells < nx;
    if (blockIdx.y & 1) {
        if (interior)
            march<T, LAW, MOB, NOISE, STAGE, -1, false, true>(P, nx, ny, pitch, k, nz, x0, j0, jend);
        else
            march<T, LAW, MOB, NOISE, STAGE, -1>(P, nx, ny, pitch, k, nz, x0, j0, jend);
    } else {
        if (interior)
            march<T, LAW, MOB, NOISE, STAGE, +1, false, true>(P, nx, ny, pitch, k, nz, x0, j0, jend);
        else
            march<T, LAW, MOB, NOISE, STAGE, +1>(P, nx, ny, pitch, k, nz, x0, j0, jend);
    }
}

template <typename T, int LAW, int MOB, int NOISE, int STAGE>
cudaError_t launch_t(const StepArgs &a, cudaStream_t st)
{
    const KV<P2<T>> k = make_kv(CoefT<T>{(T)a.k.cA, (T)a.k.cChi, (T)a.k.cG, (T)a.k.cR, (T)a.k.cN});
    NoiseT<T> nz;
    nz.seed = a.sg.seed;
    nz.step = (uint64_t)a.step;
    nz.dist = a.sg.dist;
    nz.sigma0 = (T)a.sg.sigma0;
    nz.amp = (T)a.sg.amp;
    set_noise_keys(nz);
    Ptrs<T> P{(const T *)a.b, (const T *)a.n, (const T *)a.s, (const T *)a.bu,
              (const T *)a.nu, (T *)a.bo, (T *)a.no};
    const dim3 grid((a.nx + kThreads * kCells - 1) / (kThreads * kCells),
                    (a.ny + a.rows - 1) / a.rows);
    step_kernel<T, LAW, MOB, NOISE, STAGE><<<grid, kThreads, 0, st>>>(P, a.nx, a.ny, a.pitch, k, nz,
                                                                        a.rows);
    return cudaGetLastError();
}

template <typename T, int LAW, int MOB>
cudaError_t launch_ns(const StepArgs &a, cudaStream_t st)
{
    if (a.sg.per_step)
        return a.stage ? launch_t<T, LAW, MOB, 1, 1>(a, st) : launch_t<T, LAW, MOB, 1, 0>(a, st);
    return a.stage ? launch_t<T, LAW, MOB, 0, 1>(a, st) : launch_t<T, LAW, MOB, 0, 0>(a, st);
}

template <typename T>
cudaError_t launch_prec(const StepArgs &a, cudaStream_t st)
{
    if (a.law == CX_CHEMO_RECEPTOR)
        return a.mob == CX_MOBILITY_CENTRAL ? launch_ns<T, CX_CHEMO_RECEPTOR, CX_MOBILITY_CENTRAL>(a, st)
                                            : launch_ns<T, CX_CHEMO_RECEPTOR, CX_MOBILITY_UPWIND>(a, st);
    return a.mob == CX_MOBILITY_CENTRAL ? launch_ns<T, CX_CHEMO_CONSTANT, CX_MOBILITY_CENTRAL>(a, st)
                                        : launch_ns<T, CX_CHEMO_CONSTANT, CX_MOBILITY_UPWIND>(a, st);
}

}  // namespace

cudaError_t launch_step(int prec, const StepArgs &a, cudaStream_t st)
{
    return prec == CX_PREC_F64 ? launch_prec<double>(a, st) : launch_prec<float>(a, st);
}

}  // namespace cx
