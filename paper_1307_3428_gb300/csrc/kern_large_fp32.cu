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
        const unsigned blocks = (unsigned)((cols + a.G - 1) / a.G);                \
        switch (a.stage) {                                                         \
        case LARGE_START:                                                          \
            return launch_pdl(large_col_kernel<float, LN, RR, LARGE_START>, blocks, P * a.G, \
                              smem, s, pdl, a);                                    \
        case 0:                                                                    \
            return launch_pdl(large_col_kernel<float, LN, RR, 0>, blocks, P * a.G, smem, s, \
                              pdl, a);                                             \
        case 1:                                                                    \
            return launch_pdl(large_col_kernel<float, LN, RR, 1>, blocks, P * a.G, smem, s, \
                              pdl, a);                                             \
        case 2:                                                                    \
            return launch_pdl(large_col_kernel<float, LN, RR, 2>, blocks, P * a.G, smem, s, \
                              pdl, a);                                             \
        case 3:                                                                    \
            return launch_pdl(large_col_kernel<float, LN, RR, 3>, blocks, P * a.G, smem, s, \
                              pdl, a);                                             \
        case LARGE_FINAL:                                                          \
            return launch_pdl(large_col_kernel<float, LN, RR, LARGE_FINAL>, blocks, P * a.G, \
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

#define CME_GRID_SHAPES(X) X(8, 7) X(8, 8) X(9, 8) X(9, 9)

bool large_grid_fits(int logN1, int logN2, long long blocks, int sms)
{
    switch (logN1 * 32 + logN2) {
#define CME_CASE(L1, L2)                                                                    \
    case L1 * 32 + L2: {                                                                     \
        auto k = large_grid_kernel<float, L1, L2, 8>;                                        \
        constexpr size_t smem = large_grid_smem<float, L1, L2, 8>();                          \
        if (prepare_smem(k, smem) != cudaSuccess) {                                          \
            cudaGetLastError();                                                              \
            return false;                                                                    \
        }                                                                                    \
        int per = 0;                                                                         \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, Plan<L1, 8>::P, smem) !=  \
            cudaSuccess) {                                                                   \
            cudaGetLastError();                                                              \
            return false;                                                                    \
        }                                                                                    \
        return (long long)per * sms >= blocks;                                               \
    }
        CME_GRID_SHAPES(CME_CASE)
#undef CME_CASE
    default:
        return false;
    }
}

cudaError_t launch_large_grid_fp32(int logN1, int logN2, const LargeArgs& a, long long blocks,
                                   cudaStream_t s)
{
    switch (logN1 * 32 + logN2) {
#define CME_CASE(L1, L2)                                                                    \
    case L1 * 32 + L2: {                                                                     \
        auto k = large_grid_kernel<float, L1, L2, 8>;                                        \
        constexpr size_t smem = large_grid_smem<float, L1, L2, 8>();                          \
        cudaError_t e = prepare_smem(k, smem);                                               \
        if (e != cudaSuccess)                                                                \
            return e;                                                                        \
        cudaLaunchConfig_t cfg = {};                                                         \
        cfg.gridDim = dim3((unsigned)blocks, 1, 1);                                          \
        cfg.blockDim = dim3(Plan<L1, 8>::P, 1, 1);                                           \
        cfg.dynamicSmemBytes = smem;                                                         \
        cfg.stream = s;                                                                      \
        cudaLaunchAttribute at[1];                                                           \
        at[0].id = cudaLaunchAttributeCooperative;                                           \
        at[0].val.cooperative = 1;                                                           \
        cfg.attrs = at;                                                                      \
        cfg.numAttrs = 1;                                                                    \
        return cudaLaunchKernelEx(&cfg, k, a);                                               \
    }
        CME_GRID_SHAPES(CME_CASE)
#undef CME_CASE
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace cme
