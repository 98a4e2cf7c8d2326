// Large-N (four-step) row and column kernels, FP32.
#include "cme_launch.cuh"
#include "cme_large.cuh"

namespace cme {

#define CME_LARGE_SHAPES(X) \
    X(6, 8) X(7, 8) X(8, 8) X(9, 8) X(10, 8) X(8, 4) X(9, 4) X(10, 4)

cudaError_t launch_large_row_fp32(int logN2, int R, const LargeArgs& a, long long rows,
                                  cudaStream_t s,
                                  bool pdl)
{
    switch (logN2 * 32 + R) {
#define CME_CASE(LN, RR)                                                          \
    case LN * 32 + RR: {                                                                    \
        constexpr int P = Plan<LN, RR>::P;                                        \
        const size_t smem = smem_bytes_for<float>(LN, RR, a.G);                    \
        auto k = large_row_kernel<float, LN, RR>;                                  \
        return launch_pdl(k, (unsigned)((rows + a.G - 1) / a.G), P * a.G, smem, s, pdl, a); \
    }
        CME_LARGE_SHAPES(CME_CASE)
#undef CME_CASE
    default:
        return cudaErrorInvalidValue;
    }
}

cudaError_t launch_large_col_fp32(int logN1, int R, const LargeArgs& a, long long cols,
                                  cudaStream_t s,
                                  bool pdl)
{
    switch (logN1 * 32 + R) {
#define CME_CASE(LN, RR)                                                          \
    case LN * 32 + RR: {                                                                    \
        constexpr int P = Plan<LN, RR>::P;                                        \
        const size_t smem = smem_bytes_for<float>(LN, RR, a.G);                    \
        auto k = large_col_kernel<float, LN, RR>;                                  \
        return launch_pdl(k, (unsigned)((cols + a.G - 1) / a.G), P * a.G, smem, s, pdl, a); \
    }
        CME_LARGE_SHAPES(CME_CASE)
#undef CME_CASE
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace cme
