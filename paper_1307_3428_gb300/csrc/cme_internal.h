// Shared host/device definitions of the CME library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cme {

enum { PREC_FP64 = 0, PREC_FP32 = 1 };
enum { METHOD_RK4IP = 0, METHOD_STRANG = 1 };
enum { DIAG_IDFT = 0, DIAG_DFT = 1, DIAG_RHS = 2 };

// Arguments of one uniform-N step launch.  All instances of the group share N; instance i of
// the group has its N modes at field offset base + i * N, in transform order (mu mod N).
struct StepArgs {
    int ninst;              // instances in this launch group
    int G;                  // instances per thread block
    long long base;         // first mode offset of the group
    void* hi;               // float2 / double2 field (hi part)
    void* lo;               // float2 compensation part (CME_FP32), unused for FP64
    const void* E;          // exp(L h/2) per mode                (RK4IP)
    const void* e1;         // expm1(L h/2) per mode              (RK4IP and Strang)
    const void* e2;         // expm1(L h) per mode                (RK4IP)
    const void* tw;         // twiddle table exp(2 pi i k / N), k < N
    const double2* pump;    // per-instance pump sqrt(kappa_ext) A_in (group-relative)
    const double2* cpump;   // per-instance Strang pump increment over h/2
    const double2* cpump2;  // ... over h (merged linear flows between Strang steps), or null
    const double* g0;       // per-instance Kerr coefficient g0
    int* status;            // per-instance status (group-relative)
    const int* phys;        // per-instance physical mode count M (group-relative; null: all N)
    const void* kerr;       // per-mode Kerr factors g0_mu / g0 in the field precision, laid out
                            // like E (null: every mode takes its instance's g0)
    long long nsteps;
    double h;
    float hf, hhf, h6f;     // h, h/2, h/6 rounded once to FP32 on the host
    int diag_mode;          // diagnostics kernel: DIAG_*
    void* diag_out;         // diagnostics output (same layout as the field)
    int a2a_fault;          // test of the bounded waits: cluster all-to-alls expect 8 bytes
                            // more than are sent and poll briefly (0 in normal use)
    int smem_min;           // one-block launches: at least this much dynamic shared memory
    int single_steps;       // Strang: every step on its own (no merged linear flows), as the
                            // adjoint's recomputation takes them
};

// Shared-memory footprint of one instance group (one instance of N = 2^logN handled by N/R
// threads): two padded ping-pong exchange buffers; for wide groups whose registers are scarce,
// the Runge-Kutta accumulator S and (FP32) the compensation word of the field; and, for FP32
// groups of N >= 2048 (twiddles neither in registers nor read from the global table), each
// thread's pass twiddles in thread-major order.
__host__ __device__ constexpr bool acc_in_smem(int tbytes, int logN, int R)
{
    return tbytes == 4 ? R >= 16 : logN >= 11;
}
__host__ __device__ constexpr bool twiddles_in_smem(int tbytes, int logN)
{
    return tbytes == 4 && logN >= 11;
}
__host__ __device__ constexpr int log2_radix(int R) { return R >= 16 ? 4 : R >= 8 ? 3 : R >= 4 ? 2 : 1; }
__host__ __device__ constexpr size_t xbuf_bytes(int tbytes, int logN)
{
    return (size_t)2 * (tbytes == 4 ? 1 : 2) * ((1 << logN) + (1 << logN) / 16 + 1) * 8;
}
__host__ __device__ constexpr size_t acc_bytes(int tbytes, int logN, int R)
{
    return acc_in_smem(tbytes, logN, R) ? (size_t)(1 << logN) * 2 * tbytes * (tbytes == 4 ? 2 : 1)
                                        : 0;
}
// (passes - 1) * (R - 1) twiddles per thread, N / R threads, 8-byte (FP32) complex values
__host__ __device__ constexpr size_t tw_bytes(int tbytes, int logN, int R)
{
    return twiddles_in_smem(tbytes, logN)
               ? (size_t)((logN + log2_radix(R) - 1) / log2_radix(R) - 1) * (R - 1) *
                     ((1 << logN) / R) * 8
               : 0;
}
__host__ __device__ constexpr size_t group_smem_bytes(int tbytes, int logN, int R)
{
    return xbuf_bytes(tbytes, logN) + acc_bytes(tbytes, logN, R) + tw_bytes(tbytes, logN, R);
}

// Cluster launches: one instance spread over the C blocks of a thread-block cluster.  Compiled
// for R = 8 with (log2 N, C) in {(8, 2)} (small case for tests) and {11, 12} x {2, 4, 8}.
__host__ __device__ constexpr bool cluster_shape_compiled(int logN, int R, int C)
{
    return R == 8 && ((logN == 8 && C == 2) || ((logN == 11 || logN == 12) &&
                                                (C == 2 || C == 4 || C == 8)));
}
cudaError_t launch_cluster_step_fp32(int method, int logN, int R, int C, const StepArgs& a,
                                     cudaStream_t s);
cudaError_t launch_cluster_step_fp64(int method, int logN, int R, int C, const StepArgs& a,
                                     cudaStream_t s);

// Launch one uniform-N group; implemented per precision and method in the kernel units.
cudaError_t launch_step_fp64_rk4ip(int logN, int R, const StepArgs& a, cudaStream_t s);
cudaError_t launch_step_fp64_strang(int logN, int R, const StepArgs& a, cudaStream_t s);
cudaError_t launch_step_fp32_rk4ip(int logN, int R, const StepArgs& a, cudaStream_t s);
cudaError_t launch_step_fp32_strang(int logN, int R, const StepArgs& a, cudaStream_t s);
// The same with the physical-mode mask compiled in (a.phys set); the launchers above forward
// to these when a.phys is not null.
cudaError_t launch_step_fp64_rk4ip_masked(int logN, int R, const StepArgs& a, cudaStream_t s);
cudaError_t launch_step_fp64_strang_masked(int logN, int R, const StepArgs& a, cudaStream_t s);
cudaError_t launch_step_fp32_rk4ip_masked(int logN, int R, const StepArgs& a, cudaStream_t s);
cudaError_t launch_step_fp32_strang_masked(int logN, int R, const StepArgs& a, cudaStream_t s);
cudaError_t launch_diag_fp64(int logN, int R, const StepArgs& a, cudaStream_t s);
cudaError_t launch_diag_fp32(int logN, int R, const StepArgs& a, cudaStream_t s);

// Record an error message for cme_last_error() and return `code` (cme_api.cu).
int report_error(int code, const char* fmt, ...);
// Add n to the count of kernels this library launched (cme_kernel_launches; cme_api.cu).
void count_launches(long n);
// One-block launch plan of a uniform-N group under default options: values per thread *R and
// instances per block *G, the rule cme_batch_create applies before its choice of clusters
// (cme_api.cu).  sms: the device's multiprocessor count.
void default_group_plan(int logN, int prec, int count, int sms, int* R, int* G);

// Auxiliary kernels (aux_kernels.cu).
struct PropArgs {
    int total;                // modes in the batch
    const int* mode_inst;     // instance of each mode (transform order layout)
    const double* kappa;      // per mode, transform order
    const double* omega;      // per mode, omega_mu - omega_0
    const double* sigma;      // per instance
    const double2* pump;      // per instance
    const int* inst_N;        // per instance
    const long long* inst_off;
    double h;
    int prec;
    void* E;
    void* e1;
    void* e2;
    void* e1h;                // Strang: expm1(L h/2)
    double2* cpump;           // Strang pump increment per instance
    double2* cpump2;          // the same over h (null: not computed)
    int ninst;
    double2* cphi;            // optional (null: skipped): per instance phi(L_0) and phi'(L_0),
                              // phi(L) = (exp(L h/2) - 1)/L, the factor of the Strang pump
                              // increment and its derivative (the Strang adjoint's pump terms)
};
cudaError_t launch_propagators(const PropArgs& a, cudaStream_t s);
cudaError_t launch_twiddles(int N, int prec, void* out, cudaStream_t s);
// Centred FP64 <-> internal transform-order field (optionally split into hi/lo).  inst_M (may
// be null): per-instance physical mode count; import sets the padding modes to zero.
cudaError_t launch_import(int prec, int total, const int* mode_inst, const int* inst_N,
                          const long long* inst_off, const int* inst_M, const double2* src,
                          void* hi, void* lo, cudaStream_t s);
cudaError_t launch_export(int prec, int total, const int* mode_inst, const int* inst_N,
                          const long long* inst_off, const void* hi, const void* lo,
                          double2* dst, int what, const double* omega, const double* sigma,
                          double tau, cudaStream_t s);
cudaError_t launch_export_plain(int prec, int total, const int* mode_inst, const int* inst_N,
                                const long long* inst_off, const void* src, double2* dst,
                                int reorder_centred, cudaStream_t s);
cudaError_t run_fma_peak(int prec, double* flops);
cudaError_t run_l2_peak(size_t bytes, double* bytes_per_s);

// Gradient helpers (aux_kernels.cu).
// Log-power-spectrum misfit terms (log10(|D_mu|^2 + eps) - T_mu)^2 per mode (loss_modes) and
// the cotangent dbar = dL/dRe D + i dL/dIm D in the field precision (transform order).
cudaError_t launch_loss_seed(int prec, int total, const int* mode_inst, const int* inst_N,
                             const long long* inst_off, const void* hi, const void* lo,
                             const double* target, double eps, double* loss_modes, void* dbar,
                             cudaStream_t s);
// Strang gradients: turn the accumulated cotangent cbar of each instance's pump increment
// c = phi(L_0) p (in pbar) into the pump cotangent pbar = conj(phi) cbar, and add
// conj(p phi'(L_0)) cbar to the L cotangent of the pumped mode (gL at the instance offset).
cudaError_t launch_strang_pump_grad(int count, const long long* inst_off, const double2* cphi,
                                    const double2* pump, double2* pbar, double2* gL,
                                    cudaStream_t s);
// Per instance, in a fixed summation order: red[4i..4i+3] = (sum_mu g_mu, sum g_mu mu^2/2,
// sum g_mu mu^3/6, L_i) with g_mu = Im gL_mu (the cotangent of Im L_mu = omega_mu - omega_0 -
// sigma) and L_i the instance's loss.
cudaError_t launch_grad_reduce(int count, const int* inst_N, const long long* inst_off,
                               const double2* gL, const double* loss_modes, double* red,
                               cudaStream_t s);
// Centred FP64 outputs: dD0 (complex), domega = g - delta_{mu,0} sum g, dkappa = -Re gL / 2.
cudaError_t launch_grad_export(int prec, int total, const int* mode_inst, const int* inst_N,
                               const long long* inst_off, const void* dbar, const double2* gL,
                               const double* red, double2* dD0, double* domega, double* dkappa,
                               cudaStream_t s);
struct AdjArgs;  // cme_adjoint_args.h
// C = blocks per instance (1: instances packed a.s.G per block; 2, 4, 8: thread-block cluster
// per instance, for the shapes cluster_shape_compiled accepts).
// role = ADJ_BACKWARD or ADJ_RECOMPUTE (cme_adjoint_args.h), for segment a.seg.
cudaError_t launch_adjoint_fp32(int role, int logN, int R, int C, const AdjArgs& a, cudaStream_t s);
cudaError_t launch_adjoint_fp64(int role, int logN, int R, int C, const AdjArgs& a, cudaStream_t s);
cudaError_t launch_adjoint_cluster_fp32(int role, int logN, int R, int C, const AdjArgs& a,
                                        cudaStream_t s);
cudaError_t launch_adjoint_cluster_fp64(int role, int logN, int R, int C, const AdjArgs& a,
                                        cudaStream_t s);
// The same roles for the Strang split step (a.method == METHOD_STRANG; launch_adjoint_fp32/fp64
// forward to these), C = 1 or a cluster shape.
cudaError_t launch_adjoint_strang_fp32(int role, int logN, int R, int C, const AdjArgs& a,
                                       cudaStream_t s);
cudaError_t launch_adjoint_strang_fp64(int role, int logN, int R, int C, const AdjArgs& a,
                                       cudaStream_t s);

}  // namespace cme

namespace cme {

// One persistent launch for a batch with several N: blocks of 256 threads take tiles
// (group, first instance) from a work counter, heaviest first; each tile runs the uniform
// step body of its N on 256/P instances.
constexpr int FUSED_THREADS = 256;
constexpr int MAX_GROUPS = 12;
struct FusedTile {
    int group;
    int first;   // group-relative first instance
};
struct FusedArgs {
    int ntiles;
    const FusedTile* tiles;  // heaviest first
    int* counter;            // zeroed before each launch
    int ngroups;
    int logN[MAX_GROUPS];
    StepArgs g[MAX_GROUPS];  // per group; G is the tile width 256 / P
};
// Values per thread the fused kernel uses for N = 2^logN (P = N/R <= 256).
inline int fused_radix(int logN) { return logN <= 2 ? 4 : (logN >= 12 ? 16 : 8); }
size_t fused_smem_bytes(int prec, const int* logN, int ngroups);
cudaError_t launch_fused_fp32(int method, const FusedArgs& a, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_fused_fp64(int method, const FusedArgs& a, int grid, size_t smem, cudaStream_t s);

}  // namespace cme

namespace cme {
struct LargeArgs;
// pdl = true launches with programmatic stream serialisation (cme_large.cuh: pdl_wait)  // cme_large.cuh
cudaError_t launch_large_row_fp32(int logN2, int R, const LargeArgs& a, long long rows,
                                  cudaStream_t s,
                                  bool pdl);
cudaError_t launch_large_row_fp64(int logN2, int R, const LargeArgs& a, long long rows,
                                  cudaStream_t s,
                                  bool pdl);
cudaError_t launch_large_col_fp32(int logN1, int R, const LargeArgs& a, long long cols,
                                  cudaStream_t s,
                                  bool pdl);
cudaError_t launch_large_col_fp64(int logN1, int R, const LargeArgs& a, long long cols,
                                  cudaStream_t s,
                                  bool pdl);
// The grid-barrier kernel of FP32 four-step groups at 8 values per thread (cme_large.cuh:
// large_grid_kernel), compiled for (log2 N1, log2 N2) in {(8, 7), (8, 8), (9, 8), (9, 9)}.
// large_grid_fits: whether `blocks` blocks are resident at once on `sms` SMs (the condition of
// its cooperative launch); launch_large_grid_fp32 launches a.nsteps steps as one kernel.
bool large_grid_fits(int logN1, int logN2, long long blocks, int sms);
cudaError_t launch_large_grid_fp32(int logN1, int logN2, const LargeArgs& a, long long blocks,
                                   cudaStream_t s);
}  // namespace cme
