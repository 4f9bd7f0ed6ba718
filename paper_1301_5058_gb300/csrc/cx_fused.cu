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
#include "cx_internal.h"

namespace cx {
namespace fused {
// defined in cx_fused_kernels.cuh, instantiated in cx_fused_inst.cu
template <typename T, int LAW, int MOB>
cudaError_t launch_fused_lm(const StepArgs &a, bool heun, cudaStream_t st);
}  // namespace fused

namespace {

template <typename T>
cudaError_t launch_prec(const StepArgs &a, bool heun, cudaStream_t st)
{
    if (a.law == CX_CHEMO_RECEPTOR)
        return a.mob == CX_MOBILITY_CENTRAL
                   ? fused::launch_fused_lm<T, CX_CHEMO_RECEPTOR, CX_MOBILITY_CENTRAL>(a, heun, st)
                   : fused::launch_fused_lm<T, CX_CHEMO_RECEPTOR, CX_MOBILITY_UPWIND>(a, heun, st);
    return a.mob == CX_MOBILITY_CENTRAL
               ? fused::launch_fused_lm<T, CX_CHEMO_CONSTANT, CX_MOBILITY_CENTRAL>(a, heun, st)
               : fused::launch_fused_lm<T, CX_CHEMO_CONSTANT, CX_MOBILITY_UPWIND>(a, heun, st);
}

}  // namespace

cudaError_t launch_fused(int prec, const StepArgs &a, int heun, cudaStream_t st)
{
    return prec == CX_PREC_F64 ? launch_prec<double>(a, heun != 0, st)
                               : launch_prec<float>(a, heun != 0, st);
}

}  // namespace cx
