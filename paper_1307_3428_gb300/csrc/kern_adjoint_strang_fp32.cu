// Adjoint kernels of the Strang split step, FP32: per segment, the recomputation of the states
// and Kerr-flow fields, and the backward pass; one block per instance group or one
// thread-block cluster per instance.
#include "cme_launch.cuh"
#include "cme_adjoint.cuh"

namespace cme {

template <int LN, int RR, typename KernelT>
static cudaError_t launch_strang_adj_shape(KernelT k, const AdjArgs& a, cudaStream_t s)
{
    constexpr int P = Plan<LN, RR>::P;
    const size_t smem = smem_bytes_for<float>(LN, RR, a.s.G);
    cudaError_t e = prepare_smem(k, smem);
    if (e != cudaSuccess)
        return e;
    k<<<(a.s.ninst + a.s.G - 1) / a.s.G, P * a.s.G, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_strang_fp32(int role, int logN, int R, int C, const AdjArgs& a,
                                      cudaStream_t s)
{
    if (C > 1) {
        switch ((logN * 32 + R) * 16 + C) {
#define CME_CASE(LN, RR, CC)                                                                  \
    case (LN * 32 + RR) * 16 + CC:                                                            \
        return role == ADJ_RECOMPUTE                                                          \
                   ? launch_clustered(segment_kernel<float, LN, RR, CC, METHOD_STRANG>,         \
                                      a.s.ninst * CC, Plan<LN, RR>::P / CC,                   \
                                      cluster_smem_bytes<float, LN, RR, CC>(), CC, s, a)        \
                   : launch_clustered(strang_adjoint_kernel<float, LN, RR, CC>, a.s.ninst * CC, \
                                      Plan<LN, RR>::P / CC,                                   \
                                      cluster_smem_bytes<float, LN, RR, CC>(), CC, s, a);
            CME_FOR_EACH_CLUSTER_SHAPE(CME_CASE)
#undef CME_CASE
        default:
            return cudaErrorInvalidValue;
        }
    }
    switch (logN * 32 + R) {
#define CME_CASE(LN, RR)                                                                      \
    case LN * 32 + RR:                                                                        \
        return role == ADJ_RECOMPUTE                                                          \
                   ? launch_strang_adj_shape<LN, RR>(                                         \
                         segment_kernel<float, LN, RR, 1, METHOD_STRANG>, a, s)                 \
                   : launch_strang_adj_shape<LN, RR>(strang_adjoint_kernel<float, LN, RR>, a, s);
        CME_FOR_EACH_SHAPE(CME_CASE)
#undef CME_CASE
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace cme
