// Diagnostics kernels (one transform or one right-hand side), FP64.
#include "cme_launch.cuh"

namespace cme {

cudaError_t launch_diag_fp64(int logN, int R, const StepArgs& a, cudaStream_t s)
{
    switch (logN * 32 + R) {
#define CME_CASE(LN, RR) \
    case LN * 32 + RR:   \
        return launch_diag_shape<double, LN, RR>(a, s);
        CME_FOR_EACH_SHAPE(CME_CASE)
#undef CME_CASE
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace cme
