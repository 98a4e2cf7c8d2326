// Adjoint (backward) kernels of RK4IP, FP32.
#include "cme_launch.cuh"
#include "cme_adjoint.cuh"

namespace cme {

cudaError_t launch_adjoint_fp32(int logN, int R, const AdjArgs& a, cudaStream_t s)
{
    switch (logN * 32 + R) {
#define CME_CASE(LN, RR)                                                         \
    case LN * 32 + RR: {                                                         \
        constexpr int P = Plan<LN, RR>::P;                                       \
        const size_t smem = smem_bytes_for<float>(LN, RR, a.s.G);                 \
        auto k = adjoint_kernel<float, LN, RR>;                                   \
        cudaError_t e = prepare_smem(k, smem);                                   \
        if (e != cudaSuccess)                                                    \
            return e;                                                            \
        k<<<(a.s.ninst + a.s.G - 1) / a.s.G, P * a.s.G, smem, s>>>(a);           \
        return cudaGetLastError();                                               \
    }
        CME_FOR_EACH_SHAPE(CME_CASE)
#undef CME_CASE
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace cme
