// Adjoint kernels of RK4IP, FP32: per segment, the recomputation of states and stage values
// and the backward pass.
#include "cme_launch.cuh"
#include "cme_adjoint.cuh"

namespace cme {

template <int LN, int RR, typename KernelT>
static cudaError_t launch_adj_shape(KernelT k, const AdjArgs& a, cudaStream_t s)
{
    constexpr int P = Plan<LN, RR>::P;
    const size_t smem = smem_bytes_for<float>(LN, RR, a.s.G);
    cudaError_t e = prepare_smem(k, smem);
    if (e != cudaSuccess)
        return e;
    k<<<(a.s.ninst + a.s.G - 1) / a.s.G, P * a.s.G, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_fp32(int role, int logN, int R, int C, const AdjArgs& a, cudaStream_t s)
{
    if (a.method == METHOD_STRANG)
        return launch_adjoint_strang_fp32(role, logN, R, C, a, s);
    if (C > 1)
        return launch_adjoint_cluster_fp32(role, logN, R, C, a, s);
    switch (logN * 32 + R) {
#define CME_CASE(LN, RR)                                                                  \
    case LN * 32 + RR:                                                                    \
        return role == ADJ_RECOMPUTE                                                      \
                   ? launch_adj_shape<LN, RR>(segment_kernel<float, LN, RR>, a, s)          \
                   : launch_adj_shape<LN, RR>(adjoint_kernel<float, LN, RR>, a, s);
        CME_FOR_EACH_SHAPE(CME_CASE)
#undef CME_CASE
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace cme
