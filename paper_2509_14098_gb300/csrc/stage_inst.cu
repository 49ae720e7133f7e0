// stage_inst.cu — explicit instantiation of the stage-sweep launchers for one
// (precision, direction, register width): the build compiles this file once per
// combination with SVK_INST_REAL (float / double), SVK_INST_NV (1 forward, 2 adjoint)
// and SVK_INST_R defined.
#include "stage_impl.cuh"

#if defined(SVK_INST_REAL) && defined(SVK_INST_NV) && defined(SVK_INST_R)
namespace svk {
template cudaError_t launch_R<SVK_INST_REAL, SVK_INST_R, SVK_INST_NV>(const StageLaunch&, const Stage&, cudaStream_t,
                                                                       uint32_t*);
}  // namespace svk
#endif
