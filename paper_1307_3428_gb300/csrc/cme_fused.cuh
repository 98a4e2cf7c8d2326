// One persistent launch for a batch mixing several N (the uneven batch): every block is a
// worker that takes tiles from a global counter until none are left.  A tile is up to
// 256 / P instances of one launch group, run by the same step body as the uniform kernels.
#pragma once

#include "cme_step.cuh"

namespace cme {

// Each N's body is a separate (not inlined) function so that it gets its own register
// allocation instead of sharing one with every other N's body.
// (The dynamic shared memory is named here again so that the body addresses it as shared
// memory rather than through a generic pointer.)
template <typename T, int LOGN, int R, int METHOD>
__device__ __noinline__ void fused_tile(const StepArgs* a, int first)
{
    extern __shared__ __align__(16) unsigned char smem_tile[];
    step_body<T, LOGN, R, METHOD, true, true>(*a, first, smem_tile);
}

template <typename T, int METHOD>
__global__ void __launch_bounds__(FUSED_THREADS) fused_kernel(const __grid_constant__ FusedArgs fa)
{
    __shared__ int item;
    for (;;) {
        __syncthreads();  // the previous tile is finished with `item` and the buffers
        if (threadIdx.x == 0)
            item = atomicAdd(fa.counter, 1);
        __syncthreads();
        const int it = item;
        if (it >= fa.ntiles)
            return;
        const FusedTile tl = fa.tiles[it];
        const StepArgs* a = &fa.g[tl.group];
        switch (fa.logN[tl.group]) {
#define CME_FUSED_CASE(LN, RR)                               \
    case LN:                                                 \
        fused_tile<T, LN, RR, METHOD>(a, tl.first);          \
        break;
            CME_FUSED_CASE(2, 4)
            CME_FUSED_CASE(3, 8)
            CME_FUSED_CASE(4, 8)
            CME_FUSED_CASE(5, 8)
            CME_FUSED_CASE(6, 8)
            CME_FUSED_CASE(7, 8)
            CME_FUSED_CASE(8, 8)
            CME_FUSED_CASE(9, 8)
            CME_FUSED_CASE(10, 8)
            CME_FUSED_CASE(11, 8)
            CME_FUSED_CASE(12, 16)
#undef CME_FUSED_CASE
        default:
            break;
        }
    }
}

template <typename T>
inline cudaError_t launch_fused_t(int method, const FusedArgs& a, int grid, size_t smem,
                                  cudaStream_t s)
{
    if (method == METHOD_RK4IP) {
        auto k = fused_kernel<T, METHOD_RK4IP>;
        cudaError_t e = prepare_smem(k, smem);
        if (e != cudaSuccess)
            return e;
        k<<<grid, FUSED_THREADS, smem, s>>>(a);
    } else {
        auto k = fused_kernel<T, METHOD_STRANG>;
        cudaError_t e = prepare_smem(k, smem);
        if (e != cudaSuccess)
            return e;
        k<<<grid, FUSED_THREADS, smem, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace cme
