// Instantiations of the CE kernel for the FIXED32 fold (one translation unit per
// fold mode, so that the modes compile in parallel).
#include "gce_kernel.cuh"

namespace gce {

const void *main_kernel_ptr_fixed32(int tpt, int block, bool ovl) {
    return mode_kernel_ptr<GCE_PHASE_FIXED32>(tpt, block, ovl);
}

cudaError_t launch_main_fixed32(int tpt, int block, int grid, size_t smem, const MainArgs &a,
                              cudaStream_t s) {
    return mode_launch<GCE_PHASE_FIXED32>(tpt, block, grid, smem, a, s);
}

}  // namespace gce
