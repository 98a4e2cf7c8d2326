// Launch helpers shared by the per-precision kernel translation units.
#pragma once

#include <algorithm>

#include "cme_step.cuh"

namespace cme {

// Every compiled (log2 N, values per thread) pair.  Values per thread R: 8 is the default;
// 4 and 16 are alternative launch shapes where they fit in registers without spilling, and 2
// serves single FP64 instances of N = 64, 128 (the shortest chain of FP64 instructions).
#define CME_FOR_EACH_SHAPE(X)          \
    X(2, 4)                            \
    X(3, 8)                            \
    X(4, 8) X(4, 16)                   \
    X(5, 8) X(5, 16)                   \
    X(6, 8) X(6, 4) X(6, 16) X(6, 2)   \
    X(7, 8) X(7, 4) X(7, 16) X(7, 2)   \
    X(8, 8) X(8, 4) X(8, 16)           \
    X(9, 8) X(9, 4)                    \
    X(10, 8) X(10, 4)                  \
    X(11, 8) X(11, 16)                 \
    X(12, 8) X(12, 16)

// Cluster shapes (log2 N, R, C); must agree with cluster_shape_compiled.
#define CME_FOR_EACH_CLUSTER_SHAPE(X) \
    X(8, 8, 2)                         \
    X(11, 8, 2) X(11, 8, 4) X(11, 8, 8) \
    X(12, 8, 2) X(12, 8, 4) X(12, 8, 8)

template <typename T>
inline size_t smem_bytes_for(int logN, int R, int G)
{
    return (size_t)G * group_smem_bytes(sizeof(T), logN, R);
}

template <typename KernelT>
inline cudaError_t prepare_smem(KernelT k, size_t smem)
{
    if (smem > 48 * 1024)
        return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

// Launch `blocks` blocks of `threads` threads in clusters of C blocks along x.
template <typename KernelT, typename ArgT>
inline cudaError_t launch_clustered(KernelT k, int blocks, int threads, size_t smem, int C,
                                    cudaStream_t s, const ArgT& a)
{
    cudaError_t e = prepare_smem(k, smem);
    if (e != cudaSuccess)
        return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks, 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, a);
}

// Launch with programmatic stream serialisation (pdl = true): the kernel may start before its
// predecessor in the stream has finished, and orders itself with griddepcontrol.wait.
template <typename KernelT, typename ArgT>
inline cudaError_t launch_pdl(KernelT k, unsigned blocks, unsigned threads, size_t smem,
                              cudaStream_t s, bool pdl, const ArgT& a)
{
    cudaError_t e = prepare_smem(k, smem);
    if (e != cudaSuccess)
        return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl ? at : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, a);
}

template <typename T, int LOGN, int R, int C, int METHOD>
inline cudaError_t launch_cluster_step_shape(const StepArgs& a, cudaStream_t s)
{
    static_assert(cluster_shape_compiled(LOGN, R, C), "cluster shape list");
    return launch_clustered(cluster_step_kernel<T, LOGN, R, C, METHOD>, a.ninst * C,
                            Plan<LOGN, R>::P / C, cluster_smem_bytes<T, LOGN, R, C>(), C, s, a);
}

// MASKABLE: the kernel applies the physical-mode mask of a.phys (launched when a.phys is set).
template <typename T, int LOGN, int R, int METHOD, bool MASKABLE>
inline cudaError_t launch_step_shape(const StepArgs& a, cudaStream_t s)
{
    constexpr int P = Plan<LOGN, R>::P;
    const int threads = P * a.G;
    const int blocks = (a.ninst + a.G - 1) / a.G;
    const size_t smem = std::max(smem_bytes_for<T>(LOGN, R, a.G), (size_t)a.smem_min);
    auto k = step_kernel<T, LOGN, R, METHOD, MASKABLE>;
    cudaError_t e = prepare_smem(k, smem);
    if (e != cudaSuccess)
        return e;
    k<<<blocks, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T, int LOGN, int R>
inline cudaError_t launch_diag_shape(const StepArgs& a, cudaStream_t s)
{
    constexpr int P = Plan<LOGN, R>::P;
    const int threads = P * a.G;
    const int blocks = (a.ninst + a.G - 1) / a.G;
    const size_t smem = smem_bytes_for<T>(LOGN, R, a.G);
    auto k = diag_kernel<T, LOGN, R>;
    cudaError_t e = prepare_smem(k, smem);
    if (e != cudaSuccess)
        return e;
    k<<<blocks, threads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace cme
