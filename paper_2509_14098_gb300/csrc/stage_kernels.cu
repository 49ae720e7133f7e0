// stage_kernels.cu — dispatch of the stage-sweep kernel (stage_impl.cuh) over
// precision, direction and register width; the instantiations themselves are
// compiled from stage_inst.cu, one object per (precision, direction, width).
#include "kernels.h"
#include "stage_layout.cuh"

namespace svk {

// defined (explicitly instantiated) in the stage_inst objects
template <typename Real, int R, int NV>
cudaError_t launch_R(const StageLaunch& L, const Stage& hst, cudaStream_t s, uint32_t* grid_out);

// the smaller (single-buffered) footprint: the launch never needs more than this
size_t stage_smem_bytes(int elem_bytes, const Stage& st, bool backward) {
    return smem_bytes_nb(elem_bytes, st, backward ? 2 : 1, 1);
}

template <int NV>
static cudaError_t launch_any(int elem_bytes, const StageLaunch& L, const Stage& hst, cudaStream_t s,
                              uint32_t* grid_out) {
    if (elem_bytes == 8) {
        switch (hst.R) {
            case 1: return launch_R<float, 1, NV>(L, hst, s, grid_out);
            case 2: return launch_R<float, 2, NV>(L, hst, s, grid_out);
            case 3: return launch_R<float, 3, NV>(L, hst, s, grid_out);
            case 4: return launch_R<float, 4, NV>(L, hst, s, grid_out);
            case 5: if constexpr (NV == 1) return launch_R<float, 5, NV>(L, hst, s, grid_out);
                    break;
        }
    } else {
        switch (hst.R) {
            case 1: return launch_R<double, 1, NV>(L, hst, s, grid_out);
            case 2: return launch_R<double, 2, NV>(L, hst, s, grid_out);
            case 3: return launch_R<double, 3, NV>(L, hst, s, grid_out);
            case 4: if constexpr (NV == 1) return launch_R<double, 4, NV>(L, hst, s, grid_out);
                    break;
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_stage_fwd(int elem_bytes, const StageLaunch& L, const Stage& hst, cudaStream_t s) {
    return launch_any<1>(elem_bytes, L, hst, s, nullptr);
}
cudaError_t launch_stage_bwd(int elem_bytes, const StageLaunch& L, const Stage& hst, cudaStream_t s,
                             uint32_t* grid_out) {
    return launch_any<2>(elem_bytes, L, hst, s, grid_out);
}

}  // namespace svk
