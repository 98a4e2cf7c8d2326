// Cluster step kernels (FP32): one instance per thread-block cluster, both integrators.
#include "cme_launch.cuh"

namespace cme {

cudaError_t launch_cluster_step_fp32(int method, int logN, int R, int C, const StepArgs& a,
                                      cudaStream_t s)
{
    switch ((logN * 32 + R) * 16 + C) {
#define CME_CASE(LN, RR, CC)                                                             \
    case (LN * 32 + RR) * 16 + CC:                                                       \
        return method == METHOD_RK4IP                                                    \
                   ? launch_cluster_step_shape<float, LN, RR, CC, METHOD_RK4IP>(a, s)      \
                   : launch_cluster_step_shape<float, LN, RR, CC, METHOD_STRANG>(a, s);
        CME_FOR_EACH_CLUSTER_SHAPE(CME_CASE)
#undef CME_CASE
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace cme
