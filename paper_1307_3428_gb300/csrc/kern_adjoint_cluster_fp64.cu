// Adjoint kernels of RK4IP, FP64, one instance per thread-block cluster.
#include "cme_launch.cuh"
#include "cme_adjoint.cuh"

namespace cme {

cudaError_t launch_adjoint_cluster_fp64(int role, int logN, int R, int C, const AdjArgs& a,
                                        cudaStream_t s)
{
    switch ((logN * 32 + R) * 16 + C) {
#define CME_CASE(LN, RR, CC)                                                               \
    case (LN * 32 + RR) * 16 + CC:                                                         \
        return role == ADJ_RECOMPUTE                                                       \
                   ? launch_clustered(segment_kernel<double, LN, RR, CC>, a.s.ninst * CC,     \
                                      Plan<LN, RR>::P / CC,                                \
                                      cluster_smem_bytes<double, LN, RR, CC>(), CC, s, a)     \
                   : launch_clustered(adjoint_kernel<double, LN, RR, CC>, a.s.ninst * CC,     \
                                      Plan<LN, RR>::P / CC,                                \
                                      adj_backward_smem<double, LN, RR, CC>(), CC, s, a);
        CME_FOR_EACH_CLUSTER_SHAPE(CME_CASE)
#undef CME_CASE
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace cme
