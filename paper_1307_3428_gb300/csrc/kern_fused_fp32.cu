// Persistent work-list kernel for batches with several N, FP32.
#include "cme_launch.cuh"
#include "cme_fused.cuh"

namespace cme {

cudaError_t launch_fused_fp32(int method, const FusedArgs& a, int grid, size_t smem,
                                 cudaStream_t s)
{
    return launch_fused_t<float>(method, a, grid, smem, s);
}

}  // namespace cme
