// Large-N (four-step) row and column kernels, FP64.
#include "cme_launch.cuh"
#include "cme_large.cuh"

namespace cme {

#define CME_LARGE_SHAPES(X) \
    X(6, 8) X(7, 8) X(8, 8) X(9, 8) X(10, 8) X(8, 4) X(9, 4) X(10, 4)

cudaError_t launch_large_row_fp64(int logN2, int R, const LargeArgs& a, long long rows,
                                  cudaStream_t s,
                                  bool pdl)
{
    switch (logN2 * 32 + R) {
#define CME_CASE(LN, RR)                                                          \
    case LN * 32 + RR: {                                                                    \
        constexpr int P = Plan<LN, RR>::P;                                        \
        const size_t smem = smem_bytes_for<double>(LN, RR, a.G);                    \
        auto k = large_row_kernel<double, LN, RR>;                                  \
        return launch_pdl(k, (unsigned)((rows + a.G - 1) / a.G), P * a.G, smem, s, pdl, a); \
    }
        CME_LARGE_SHAPES(CME_CASE)
#undef CME_CASE
    default:
        return cudaErrorInvalidValue;
    }
}

cudaError_t launch_large_col_fp64(int logN1, int R, const LargeArgs& a, long long cols,
                                  cudaStream_t s,
                                  bool pdl)
{
    switch (logN1 * 32 + R) {
#define CME_CASE(LN, RR)                                                          \
    case LN * 32 + RR: {                                                                    \
        constexpr int P = Plan<LN, RR>::P;                                        \
        const size_t smem = smem_bytes_for<double>(LN, RR, a.G);                    \
        const unsigned blocks = (unsigned)((cols + a.G - 1) / a.G);                \
        switch (a.stage) {                                                         \
        case LARGE_START:                                                          \
            return launch_pdl(large_col_kernel<double, LN, RR, LARGE_START>, blocks, P * a.G, \
                              smem, s, pdl, a);                                    \
        case 0:                                                                    \
            return launch_pdl(large_col_kernel<double, LN, RR, 0>, blocks, P * a.G, smem, s, \
                              pdl, a);                                             \
        case 1:                                                                    \
            return launch_pdl(large_col_kernel<double, LN, RR, 1>, blocks, P * a.G, smem, s, \
                              pdl, a);                                             \
        case 2:                                                                    \
            return launch_pdl(large_col_kernel<double, LN, RR, 2>, blocks, P * a.G, smem, s, \
                              pdl, a);                                             \
        case 3:                                                                    \
            return launch_pdl(large_col_kernel<double, LN, RR, 3>, blocks, P * a.G, smem, s, \
                              pdl, a);                                             \
        case LARGE_FINAL:                                                          \
            return launch_pdl(large_col_kernel<double, LN, RR, LARGE_FINAL>, blocks, P * a.G, \
                              smem, s, pdl, a);                                    \
        default:                                                                   \
            return cudaErrorInvalidValue;                                          \
        }                                                                          \
    }
        CME_LARGE_SHAPES(CME_CASE)
#undef CME_CASE
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace cme
