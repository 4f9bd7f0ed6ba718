// cx_batch_inst.cu -- explicit instantiations of the batch step kernels
// (cx_batch_kernels.cuh).  The build compiles this file once per
// (precision, chemotaxis law, mobility), given as CX_INST_PREC (0 FP64,
// 1 FP32), CX_INST_LAW and CX_INST_MOB, so that the eight sets of kernels
// compile in parallel; without the macros it instantiates all of them.
#include "cx_batch_kernels.cuh"

namespace cx {
namespace batch {

#define CX_BATCH_INST(T, LAW, MOB)                                                             \
    template cudaError_t launch_step_lm<T, LAW, MOB>(const void *, const int4 *, int, int, int, \
                                                     int, int, const long long *, int,         \
                                                     cudaStream_t);                            \
    template cudaError_t launch_fused_lm<T, LAW, MOB>(const void *, const int4 *, int, int,     \
                                                      int, int, int, const long long *, int,   \
                                                      cudaStream_t);                           \
    template cudaError_t launch_resident_lm<T, LAW, MOB>(const void *, const int4 *, int, int,  \
                                                         int, int, int, int, void *, long long, \
                                                         const long long *, int, cudaStream_t);

#if defined(CX_INST_PREC) && defined(CX_INST_LAW) && defined(CX_INST_MOB)
#if CX_INST_PREC == 0
CX_BATCH_INST(double, CX_INST_LAW, CX_INST_MOB)
#else
CX_BATCH_INST(float, CX_INST_LAW, CX_INST_MOB)
#endif
#else
CX_BATCH_INST(float, CX_CHEMO_RECEPTOR, CX_MOBILITY_CENTRAL)
CX_BATCH_INST(float, CX_CHEMO_RECEPTOR, CX_MOBILITY_UPWIND)
CX_BATCH_INST(float, CX_CHEMO_CONSTANT, CX_MOBILITY_CENTRAL)
CX_BATCH_INST(float, CX_CHEMO_CONSTANT, CX_MOBILITY_UPWIND)
CX_BATCH_INST(double, CX_CHEMO_RECEPTOR, CX_MOBILITY_CENTRAL)
CX_BATCH_INST(double, CX_CHEMO_RECEPTOR, CX_MOBILITY_UPWIND)
CX_BATCH_INST(double, CX_CHEMO_CONSTANT, CX_MOBILITY_CENTRAL)
CX_BATCH_INST(double, CX_CHEMO_CONSTANT, CX_MOBILITY_UPWIND)
#endif

}  // namespace batch
}  // namespace cx
