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
    const double* g0;       // per-instance Kerr coefficient g0
    int* status;            // per-instance status (group-relative)
    long long nsteps;
    double h;
    float hf, hhf, h6f;     // h, h/2, h/6 rounded once to FP32 on the host
    int diag_mode;          // diagnostics kernel: DIAG_*
    void* diag_out;         // diagnostics output (same layout as the field)
};

// Launch one uniform-N group; implemented per precision and method in the kernel units.
cudaError_t launch_step_fp64_rk4ip(int logN, int R, const StepArgs& a, cudaStream_t s);
cudaError_t launch_step_fp64_strang(int logN, int R, const StepArgs& a, cudaStream_t s);
cudaError_t launch_step_fp32_rk4ip(int logN, int R, const StepArgs& a, cudaStream_t s);
cudaError_t launch_step_fp32_strang(int logN, int R, const StepArgs& a, cudaStream_t s);
cudaError_t launch_diag_fp64(int logN, int R, const StepArgs& a, cudaStream_t s);
cudaError_t launch_diag_fp32(int logN, int R, const StepArgs& a, cudaStream_t s);

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
    int ninst;
};
cudaError_t launch_propagators(const PropArgs& a, cudaStream_t s);
cudaError_t launch_twiddles(int N, int prec, void* out, cudaStream_t s);
// Centred FP64 <-> internal transform-order field (optionally split into hi/lo).
cudaError_t launch_import(int prec, int total, const int* mode_inst, const int* inst_N,
                          const long long* inst_off, const double2* src, void* hi, void* lo,
                          cudaStream_t s);
cudaError_t launch_export(int prec, int total, const int* mode_inst, const int* inst_N,
                          const long long* inst_off, const void* hi, const void* lo,
                          double2* dst, int what, const double* omega, const double* sigma,
                          double tau, cudaStream_t s);
cudaError_t launch_export_plain(int prec, int total, const int* mode_inst, const int* inst_N,
                                const long long* inst_off, const void* src, double2* dst,
                                int reorder_centred, cudaStream_t s);
cudaError_t run_fma_peak(int prec, double* flops);

}  // namespace cme
