// Instantiations of the CE kernel for the FIXED32 fold with 1 trial per
// thread (one translation unit per fold mode and trials per thread, so that
// they compile in parallel).
#include "gce_kernel.cuh"

namespace gce {

const void *main_kernel_ptr_fixed32_t1(int block, int kv) {
    return kernel_for_variant<GCE_PHASE_FIXED32, 1>(block, kv);
}

cudaError_t launch_main_fixed32_t1(int block, int grid, size_t smem, const MainArgs &a,
                                  cudaStream_t s) {
    return launch_for_block<GCE_PHASE_FIXED32, 1>(block, grid, smem, a, s);
}

}  // namespace gce
