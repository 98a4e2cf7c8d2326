// cme_rk4ip_noalloc: the FP64 RK4IP integration of a uniform-N set of instances with every
// piece of scratch memory taken from one statically sized device array instead of cudaMalloc.
//
// Who needs this: code that is not allowed to allocate device memory itself -- for example a
// host application whose device memory all comes from its own fixed-size pool, or code that
// runs between other asynchronous work where cudaMalloc (which can synchronise the whole device)
// must not be called.  Such callers pass device pointers to the inputs and to the field; the
// internal work arrays (transform-order field, propagators, twiddles, per-instance constants,
// status words) live in g_noalloc_scratch below.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "cme.h"
#include "cme_internal.h"

namespace {

// The whole scratch area of cme_rk4ip_noalloc.  Every GPU that loads this library reserves it
// until the process exits.
constexpr size_t kScratchBytes = (size_t)CME_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch per device ordinal.  In host code the array's name is a
// host-side stand-in, not a device address, so the address must come from
// cudaGetSymbolAddress, taken once per device with that device current.  The cached address
// belongs to the device's context as it was then: after cudaDeviceReset it is stale.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

cudaError_t scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= kMaxDevices)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

// Carves 256-byte-aligned pieces off the scratch area.
struct Carver {
    unsigned char* base;
    size_t used = 0;
    void* take(size_t bytes)
    {
        void* p = base + used;
        used += (bytes + 255) / 256 * 256;
        return p;
    }
};

// Per-mode and per-instance tables in the layout the step kernels expect: transform-order
// kappa and omega - omega_0, mode -> instance map, offsets, pump sqrt(kappa_ext) A_in, g0,
// sigma; the status words start at zero.
__global__ void noalloc_tables_kernel(int N, int count, const double* kappa_c,
                                      const double* omega_c, const double* inst, double* kappa_t,
                                      double* omega_t, int* mode_inst, int* inst_N,
                                      long long* inst_off, double* sigma, double2* pump,
                                      double* g0, int* status)
{
    const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)N * count;
    if (m < total) {
        const int i = (int)(m / N);
        const int pm = (int)(m - (long long)i * N);
        const int c = (pm + N / 2) & (N - 1);
        const long long o = (long long)i * N;
        kappa_t[m] = kappa_c[o + c];
        omega_t[m] = omega_c[o + c] - omega_c[o + N / 2];
        mode_inst[m] = i;
    }
    if (m < count) {
        const double* p = inst + 5 * m;
        inst_N[m] = N;
        inst_off[m] = m * N;
        g0[m] = p[0];
        const double sk = sqrt(p[1]);
        pump[m] = make_double2(sk * p[2], sk * p[3]);
        sigma[m] = p[4];
        status[m] = 0;
    }
}

bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

}  // namespace

extern "C" int cme_rk4ip_noalloc(int N, int count, double h, long nsteps, const double* d_kappa,
                                 const double* d_omega, const double* d_inst, double* d_field,
                                 void* cuda_stream)
{
    using namespace cme;
    if (!pow2(N) || N < 4 || N > 4096)
        return report_error(CME_ERR_UNSUPPORTED_N,
                            "cme_rk4ip_noalloc: N=%d is not a power of two in [4, 4096]", N);
    if (count <= 0 || !(h > 0.0) || !std::isfinite(h) || nsteps < 0 || !d_kappa || !d_omega ||
        !d_inst || !d_field)
        return report_error(CME_ERR_INVALID_ARG, "cme_rk4ip_noalloc: invalid argument");
    const size_t total = (size_t)N * count;
    // bytes needed: field 16, propagators 48, kappa/omega 16, mode map 4 per mode; per instance
    // pump + Strang increment 32, g0 + sigma 16, N + offset 12, status 4; twiddles 16 N;
    // plus alignment padding of each of the 16 pieces
    const size_t need = total * (16 + 48 + 16 + 4) + (size_t)count * (32 + 16 + 12 + 4) +
                        (size_t)N * 16 + 16 * 256;
    if (need > kScratchBytes)
        return report_error(CME_ERR_INVALID_ARG,
                            "cme_rk4ip_noalloc: %d instances of N=%d need %zu bytes of scratch, "
                            "more than its fixed %zu bytes (use cme_batch_create/cme_step)",
                            count, N, need, kScratchBytes);
    void* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess)
        return report_error(CME_ERR_CUDA, "cme_rk4ip_noalloc: cudaGetSymbolAddress: %s",
                            cudaGetErrorString(e));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    Carver cv{(unsigned char*)base};
    double2* hi = (double2*)cv.take(total * 16);
    void* E = cv.take(total * 16);
    void* e1 = cv.take(total * 16);
    void* e2 = cv.take(total * 16);
    double* kappa_t = (double*)cv.take(total * 8);
    double* omega_t = (double*)cv.take(total * 8);
    int* mode_inst = (int*)cv.take(total * 4);
    int* inst_N = (int*)cv.take((size_t)count * 4);
    long long* inst_off = (long long*)cv.take((size_t)count * 8);
    double* sigma = (double*)cv.take((size_t)count * 8);
    double2* pump = (double2*)cv.take((size_t)count * 16);
    double2* cpump = (double2*)cv.take((size_t)count * 16);
    double* g0 = (double*)cv.take((size_t)count * 8);
    int* status = (int*)cv.take((size_t)count * 4);
    void* tw = cv.take((size_t)N * 16);

    const int threads = 256;
    const long long blocks = ((long long)total + threads - 1) / threads;
    noalloc_tables_kernel<<<(unsigned)blocks, threads, 0, s>>>(N, count, d_kappa, d_omega, d_inst,
                                                                kappa_t, omega_t, mode_inst,
                                                                inst_N, inst_off, sigma, pump, g0,
                                                                status);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = launch_twiddles(N, PREC_FP64, tw, s);
    if (e == cudaSuccess) {
        PropArgs p{};
        p.total = (int)total;
        p.mode_inst = mode_inst;
        p.kappa = kappa_t;
        p.omega = omega_t;
        p.sigma = sigma;
        p.pump = pump;
        p.inst_N = inst_N;
        p.inst_off = inst_off;
        p.h = h;
        p.prec = PREC_FP64;
        p.E = E;
        p.e1 = e1;
        p.e2 = e2;
        p.cpump = cpump;
        p.ninst = count;
        e = launch_propagators(p, s);
    }
    if (e == cudaSuccess)
        e = launch_import(PREC_FP64, (int)total, mode_inst, inst_N, inst_off, nullptr,
                          (const double2*)d_field, hi, nullptr, s);
    if (e == cudaSuccess && nsteps > 0) {
        int logN = 0;
        while ((1 << logN) < N)
            ++logN;
        // values per thread and instances per block: the one-block plan cme_batch_create
        // chooses under default options (for small sets 4 values per thread, for instance)
        int dev = 0, sms = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        int R = 8, G = 1;
        default_group_plan(logN, PREC_FP64, count, sms, &R, &G);
        StepArgs a{};
        a.ninst = count;
        a.G = G;
        a.base = 0;
        a.hi = hi;
        a.lo = nullptr;
        a.E = E;
        a.e1 = e1;
        a.e2 = e2;
        a.tw = tw;
        a.pump = pump;
        a.cpump = cpump;
        a.g0 = g0;
        a.status = status;
        a.nsteps = nsteps;
        a.h = h;
        a.hf = (float)h;
        a.hhf = (float)(0.5 * h);
        a.h6f = (float)(h / 6.0);
        if (e == cudaSuccess)
            e = launch_step_fp64_rk4ip(logN, R, a, s);
    }
    if (e == cudaSuccess)
        e = launch_export(PREC_FP64, (int)total, mode_inst, inst_N, inst_off, hi, nullptr,
                          (double2*)d_field, 1, omega_t, sigma, 0.0, s);
    // tables, twiddles, propagators, import, (step,) export
    count_launches(nsteps > 0 ? 6 : 5);
    if (e != cudaSuccess)
        return report_error(CME_ERR_CUDA, "cme_rk4ip_noalloc: launch: %s", cudaGetErrorString(e));
    return CME_OK;
}
