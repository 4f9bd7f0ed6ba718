// cx_fused_inst.cu -- explicit instantiations of the two-stage pass
// (cx_fused_kernels.cuh).  The build compiles this file once per
// (precision, chemotaxis law, mobility), given as CX_INST_PREC (0 FP64,
// 1 FP32), CX_INST_LAW and CX_INST_MOB, so that the eight sets of kernels
// compile in parallel; without the macros it instantiates all of them.
#include "cx_fused_kernels.cuh"

namespace cx {
namespace fused {

#define CX_FUSED_INST(T, LAW, MOB) \
    template cudaError_t launch_fused_lm<T, LAW, MOB>(const StepArgs &, bool, cudaStream_t);

#if defined(CX_INST_PREC) && defined(CX_INST_LAW) && defined(CX_INST_MOB)
#if CX_INST_PREC == 0
CX_FUSED_INST(double, CX_INST_LAW, CX_INST_MOB)
#else
CX_FUSED_INST(float, CX_INST_LAW, CX_INST_MOB)
#endif
#else
CX_FUSED_INST(float, CX_CHEMO_RECEPTOR, CX_MOBILITY_CENTRAL)
CX_FUSED_INST(float, CX_CHEMO_RECEPTOR, CX_MOBILITY_UPWIND)
CX_FUSED_INST(float, CX_CHEMO_CONSTANT, CX_MOBILITY_CENTRAL)
CX_FUSED_INST(float, CX_CHEMO_CONSTANT, CX_MOBILITY_UPWIND)
CX_FUSED_INST(double, CX_CHEMO_RECEPTOR, CX_MOBILITY_CENTRAL)
CX_FUSED_INST(double, CX_CHEMO_RECEPTOR, CX_MOBILITY_UPWIND)
CX_FUSED_INST(double, CX_CHEMO_CONSTANT, CX_MOBILITY_CENTRAL)
CX_FUSED_INST(double, CX_CHEMO_CONSTANT, CX_MOBILITY_UPWIND)
#endif

}  // namespace fused
}  // namespace cx
