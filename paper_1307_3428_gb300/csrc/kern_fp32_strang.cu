// STRANG step kernels, FP32: explicit instantiations and the shape dispatch.
#include "cme_launch.cuh"

namespace cme {

cudaError_t launch_step_fp32_strang(int logN, int R, const StepArgs& a, cudaStream_t s)
{
    if (a.phys || a.kerr)   // padding modes or per-mode Kerr factors in the group
        return launch_step_fp32_strang_masked(logN, R, a, s);
    switch (logN * 32 + R) {
#define CME_CASE(LN, RR) \
    case LN * 32 + RR:   \
        return launch_step_shape<float, LN, RR, METHOD_STRANG, false>(a, s);
        CME_FOR_EACH_SHAPE(CME_CASE)
#undef CME_CASE
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace cme
