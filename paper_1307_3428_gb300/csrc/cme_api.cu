// Host side of the C ABI declared in include/cme.h: instances, batches, device memory, launch
// planning, CUDA graph caching and error reporting.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "cme.h"
#include "cme_internal.h"
#include "cme_adjoint_args.h"
#include "cme_large.cuh"

using namespace cme;

namespace {

thread_local std::string g_err;
std::atomic<long> g_launches{0};

std::mutex g_alloc_mu;
cme_alloc_fn g_alloc = nullptr;
cme_free_fn g_free = nullptr;
void* g_alloc_ctx = nullptr;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

}  // namespace

int cme::report_error(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

namespace {

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(e == cudaErrorMemoryAllocation ? CME_ERR_OOM : CME_ERR_CUDA, "%s: %s (%s)", what,
                cudaGetErrorName(e), cudaGetErrorString(e));
}

#define CME_CUDA(call, what)                     \
    do {                                         \
        cudaError_t e_ = (call);                 \
        if (e_ != cudaSuccess)                   \
            return cuda_fail(e_, what);          \
    } while (0)

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
int ilog2i(int n)
{
    int l = 0;
    while ((1 << l) < n)
        ++l;
    return l;
}

// Device allocation through the registered hooks (else cudaMalloc).
void* dev_alloc(size_t bytes)
{
    if (bytes == 0)
        bytes = 16;
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    if (g_alloc)
        return g_alloc(bytes, g_alloc_ctx);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}
void dev_free(void* p, cme_free_fn f, void* ctx)
{
    if (!p)
        return;
    if (f)
        f(p, ctx);
    else
        cudaFree(p);
}

// Compiled launch shapes (values per thread R for each log2 N); must match the kernel units.
bool shape_compiled(int logN, int R)
{
    static const int shapes[][2] = {{2, 4},  {3, 8},  {4, 8},  {4, 16}, {5, 8},  {5, 16},
                                    {6, 8},  {6, 4},  {6, 16}, {6, 2},  {7, 8},  {7, 4},
                                    {7, 16}, {7, 2},  {8, 8},  {8, 4},  {8, 16}, {9, 8},
                                    {9, 4},  {10, 8}, {10, 4}, {11, 8}, {11, 16}, {12, 8},
                                    {12, 16}};
    for (auto& s : shapes)
        if (s[0] == logN && s[1] == R)
            return true;
    return false;
}

// Values per thread: 8 (N = 4: 4), except FP32 N >= 2048, which take 16: with their twiddles
// in shared memory and their propagators in registers that measured 11.7 against 13.3 us per
// step at N = 4096 and 7.2 against 7.4 at N = 2048 (GB300).
// FP64 groups too small to give every SM a warp at 8 values per thread take 4: each thread's
// chain of FP64 instructions (1/64 of the FP32 rate) then sets the step time, and halving it
// measured 31 against 55 us per step for one N = 64 instance.  Groups of N = 64 or 128 that
// hold at most one warp per SM at 2 values per thread take 2, halving the chain again: 19.4
// against 31 us per step for one N = 64 instance.  sms = 0: no such information.
int default_radix(int logN, int prec, int count = 0, int sms = 0)
{
    if (logN <= 2)
        return 4;
    if (prec == PREC_FP32 && logN >= 11)
        return 16;
    if (prec == PREC_FP64 && sms > 0 && shape_compiled(logN, 2) &&
        (long long)count * ((1 << logN) / 2) <= 32LL * sms)
        return 2;
    if (prec == PREC_FP64 && sms > 0 && shape_compiled(logN, 4) &&
        (long long)count * ((1 << logN) / 8) < 32LL * sms)
        return 4;
    return 8;
}

}  // namespace

struct cme_instance_s {
    int N = 0;
    int M = 0;   // physical modes (0: all N)
    std::vector<double> kappa, omega, field;
    std::vector<double> g0mu;   // per-mode Kerr coefficients (centred); empty: g0 on every mode
    double g0 = 0, kappa_ext = 0, ain_re = 0, ain_im = 0, sigma = 0;
};

namespace {
struct LaunchGroup {
    int logN = 0, N = 0;
    int first = 0, count = 0;   // instances [first, first+count)
    long long base = 0;         // first mode offset
    int R = 8, G = 1;
    int C = 1;                  // blocks per instance (thread-block cluster when > 1)
    bool masked = false;        // some instance has padding modes (M < N)
    bool kerr = false;          // some instance has per-mode Kerr coefficients
    // N > 4096: four-step split N = N1 N2 (column length N1, row length N2)
    bool large = false;
    int logN1 = 0, logN2 = 0, G1 = 1, G2 = 1;
    int RL = 8;                 // values per thread of the row and column kernels
    void* Y = nullptr;          // [count][N] inter-pass buffers
    void* Z = nullptr;
    bool grid = false;          // one grid-barrier kernel per call (large_grid_kernel)
    unsigned long long* bar = nullptr;   // its barrier counter
    cudaGraphExec_t chunk = nullptr;   // LARGE_CHUNK steps, replayed by cme_step
    double chunk_h = 0.0;
};
constexpr int LARGE_CHUNK = 32;
}  // namespace

struct cme_batch_s {
    int a2a_fault = 0;   // cme_debug_fault
    int count = 0;
    long long total = 0;
    cme_options opt{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int prec = PREC_FP64, method = METHOD_RK4IP;
    size_t elem = 16;  // bytes per complex field element

    // device memory
    std::vector<void*> allocs;
    cme_free_fn free_fn = nullptr;
    void* free_ctx = nullptr;
    void *hi = nullptr, *lo = nullptr, *E = nullptr, *e1 = nullptr, *e2 = nullptr,
         *diag = nullptr;
    double *kappa = nullptr, *omega = nullptr, *sigma_d = nullptr, *g0_d = nullptr;
    double2 *pump_d = nullptr, *cpump_d = nullptr, *cpump2_d = nullptr, *stage = nullptr;
    double2* cphi_d = nullptr;   // per instance phi(L_0), phi'(L_0) of the Strang pump increment
    int *mode_inst = nullptr, *inst_N = nullptr, *status_d = nullptr;
    int* phys_d = nullptr;   // per-instance physical mode count M
    void* kerr_d = nullptr;  // per-mode Kerr factors (field precision), if any instance has them
    long long* inst_off = nullptr;
    std::map<int, void*> tw;  // per log2 N

    // host copies
    std::vector<int> N_h;
    std::vector<long long> off_h;
    std::vector<double> sigma_h;
    std::vector<LaunchGroup> groups;

    double h_cur = 0.0;   // h of the current propagators (0 = none)
    double tau = 0.0;

    std::map<std::pair<double, long>, std::pair<cudaGraphExec_t, int>> graphs;

    // launch plan: 1 = one kernel per group (concurrent side streams when there are several
    // groups), 2 = one persistent work-list kernel over all groups
    int mode = 1;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> ev;      // ev[0] fork, ev[1 + i] join of side stream i
    FusedTile* tiles_d = nullptr;
    std::vector<double> sqk_h;        // sqrt(kappa_ext) per instance

    // gradient scratch (allocated by the first cme_grad call, grown when needed)
    long long g_S = 0, g_K = 0;      // checkpoints and steps per segment the scratch holds
    long long g_slots = 0;           // segments of per-step data the scratch holds
    long long grad_budget = -1;      // cme_set_grad_memory: -1 automatic, 0 never store
    void *g_ckpt_hi = nullptr, *g_ckpt_lo = nullptr, *g_stages = nullptr, *g_dbar = nullptr;
    cudaStream_t g_side = nullptr;              // recomputation stream of cme_grad
    cudaEvent_t g_ev[4] = {};                   // fork, recomputed, backward done (x2)
    double2 *g_gL = nullptr, *g_pbar = nullptr, *g_dD0 = nullptr;
    double *g_loss = nullptr, *g_red = nullptr, *g_target = nullptr, *g_domega = nullptr,
           *g_dkappa = nullptr;
    std::vector<void*> g_allocs;
    int* counter_d = nullptr;
    int ntiles = 0;
    int sms = 0;
    int smem_optin = 0;   // largest dynamic shared memory of one block

    void clear_graphs()
    {
        for (auto& kv : graphs)
            cudaGraphExecDestroy(kv.second.first);
        graphs.clear();
        for (auto& g : groups) {
            if (g.chunk)
                cudaGraphExecDestroy(g.chunk);
            g.chunk = nullptr;
        }
    }
    bool has_large() const
    {
        for (auto& g : groups)
            if (g.large)
                return true;
        return false;
    }
    void* S_large = nullptr;   // Runge-Kutta accumulator of four-step groups (per mode)

    void* alloc(size_t bytes)
    {
        void* p = dev_alloc(bytes);
        if (p)
            allocs.push_back(p);
        return p;
    }
};

namespace {

// Instances per block of a per-group kernel with R values per thread (G = 0: library choice).
int inst_per_block(int N, int R, int G, int count)
{
    const int P = N / R;
    if (G == 0)
        G = P >= 64 ? 1 : std::max(1, 64 / P);
    G = std::min(G, std::max(1, 256 / P));
    if (P >= 64)
        return 1;   // kernels for groups of >= 64 threads are compiled for one instance per block
    if (P < 32) {
        // groups narrower than a warp synchronise with __syncwarp over full warps: make the
        // block a whole number of warps (surplus groups recompute the last instance and store
        // nothing), and no more warps than the instances fill
        const int per_warp = 32 / P;
        const int g = std::min(G, std::max(count, 1));
        return (g + per_warp - 1) / per_warp * per_warp;
    }
    return std::min(G, count);
}

// (Re)compute the launch plan of every group from the options: values per thread R and
// instances per block G of the per-group kernels, and the persistent work-list tiles.
int plan_batch(cme_batch b, const cme_options& o)
{
    if (o.steps_per_launch < 0 || o.inst_per_cta < 0 || o.radix < 0 || o.persistent < 0 ||
        o.persistent > 2 || !(o.cluster == 0 || o.cluster == 1 || o.cluster == 2 ||
                              o.cluster == 4 || o.cluster == 8))
        return fail(CME_ERR_INVALID_ARG, "launch plan: invalid option");
    bool any_large = false;
    for (auto& g : b->groups) {
        if (g.large) {
            // rows of N2 and columns of N1 values, RL per thread (8, or 4 on request where
            // compiled: N1, N2 in 2^8 ... 2^10); whole warps per block
            g.RL = (o.radix == 4 && g.logN2 >= 8 && g.logN1 <= 10) ? 4 : 8;
            auto blocks_of = [&g](int len) {
                const int P = len / g.RL;
                return P >= 64 ? 1 : std::max(1, 64 / P);
            };
            g.G1 = blocks_of(1 << g.logN1);
            g.G2 = blocks_of(1 << g.logN2);
            // persistent = 2: one grid-barrier kernel per call, where all its blocks (one
            // per column) are resident at once.  Not the default: on N = 2^17 it measured
            // 35.4 against 34.8 us per step for the kernel sequence with dependent launch
            // (the barriers' fences wait for the strided stores as the kernel exits do)
            g.grid = b->prec == PREC_FP32 && g.RL == 8 && o.persistent == 2 &&
                     large_grid_fits(g.logN1, g.logN2, (long long)g.count << g.logN2, b->sms);
            any_large = true;
            continue;
        }
        int R = o.radix ? o.radix : default_radix(g.logN, b->prec, g.count, b->sms);
        // an explicit cluster request without an explicit radix takes the clusters' 8 values
        // per thread
        if (!o.radix && o.cluster > 1 && cluster_shape_compiled(g.logN, 8, o.cluster))
            R = 8;
        if (R > g.N)
            R = g.N;
        if (!shape_compiled(g.logN, R))
            return fail(CME_ERR_INVALID_ARG, "launch plan: radix %d not available for N=%d", R, g.N);
        g.R = R;
        g.G = inst_per_block(g.N, R, o.inst_per_cta, g.count);
        // blocks per instance: explicit here; the library's choice follows below
        g.C = 1;
        if (o.cluster > 1 && cluster_shape_compiled(g.logN, R, o.cluster))
            g.C = o.cluster;
    }
    // Library choice of clusters (o.cluster == 0).  Only where one block per instance leaves
    // SMs idle: the batch's one-block plan occupies at most 2/3 of the SMs.  A group of
    // N = 2048 or 4096 then takes the largest cluster whose blocks, with the other groups',
    // stay within ~3.4 per SM (all resident at once), at 8 values per thread: C = 8 in FP32
    // (C = 4 and 2 lose to one block there), C = 8, 4 or 2 in FP64.  Measured per RK4IP step,
    // FP32 N = 4096: 16 instances 11.5 -> 5.9 us, 64 instances 11.7 -> 8.2 us, 96 instances
    // 11.7 -> 15.5 us (not all blocks resident); FP64 N = 4096: 16 instances 437 -> 115 us,
    // 96 instances 437 -> 349 us (C = 4).  Mixed batches whose one-block plan fills the GPU
    // (N = 256 ... 4096 x 64) keep one block per instance: 584 ms per run, against 776 ms with
    // 8-block clusters.
    if (o.cluster == 0 && !any_large && o.persistent != 2) {   // the work-list kernel has no clusters
        long long blocks1 = 0;
        for (const auto& g : b->groups)
            blocks1 += (g.count + g.G - 1) / g.G;
        const long long cap = (long long)b->sms * 17 / 5;
        if (3 * blocks1 <= 2LL * b->sms) {
            for (auto& g : b->groups) {
                if (!(g.logN == 11 || g.logN == 12) || (o.radix && o.radix != 8))
                    continue;
                const long long others = blocks1 - (g.count + g.G - 1) / g.G;
                for (int c : {8, 4, 2}) {
                    if (b->prec == PREC_FP32 && c < 8)
                        break;
                    if (cluster_shape_compiled(g.logN, 8, c) && others + (long long)g.count * c <= cap) {
                        g.C = c;
                        g.R = 8;
                        g.G = 1;
                        break;
                    }
                }
            }
        }
    }
    // library choice: one kernel per N group on concurrent streams (measured ahead of the
    // work-list kernel on the uneven N = 256 ... 4096 workload: 1.13 s against 1.22 s)
    int mode = o.persistent;
    if (mode == 0)
        mode = 1;
    if (any_large)
        mode = 1;   // four-step groups run their own kernel sequence
    if (mode == 2) {
        // tiles of 256 / P instances (the fused kernel's own values per thread), heaviest first;
        // a tile's time scales with R log2 N
        std::vector<std::pair<int, FusedTile>> tiles;
        for (int gi = 0; gi < (int)b->groups.size(); ++gi) {
            const auto& g = b->groups[gi];
            const int Rf = fused_radix(g.logN), Pf = g.N / Rf;
            const int Gf = std::max(1, FUSED_THREADS / Pf);
            for (int f = 0; f < g.count; f += Gf)
                tiles.push_back({Rf * g.logN, FusedTile{gi, f}});
        }
        std::stable_sort(tiles.begin(), tiles.end(),
                         [](const auto& x, const auto& y) { return x.first > y.first; });
        std::vector<FusedTile> t(tiles.size());
        for (size_t i = 0; i < tiles.size(); ++i)
            t[i] = tiles[i].second;
        b->ntiles = (int)t.size();
        CME_CUDA(cudaMemcpyAsync(b->tiles_d, t.data(), t.size() * sizeof(FusedTile),
                                 cudaMemcpyHostToDevice, b->stream),
                 "launch plan: tiles");
        CME_CUDA(cudaStreamSynchronize(b->stream), "launch plan: tiles");
    }
    b->mode = mode;
    b->opt.radix = o.radix;
    b->opt.inst_per_cta = o.inst_per_cta;
    b->opt.steps_per_launch = o.steps_per_launch;
    b->opt.use_graph = o.use_graph;
    b->opt.persistent = mode;
    b->opt.cluster = o.cluster;
    b->clear_graphs();
    return CME_OK;
}

}  // namespace

void cme::count_launches(long n) { g_launches += n; }

void cme::default_group_plan(int logN, int prec, int count, int sms, int* R, int* G)
{
    const int r = std::min(default_radix(logN, prec, count, sms), 1 << logN);
    *R = r;
    *G = inst_per_block(1 << logN, r, 0, count);
}

// ------------------------------------------------------------------------------------------
extern "C" {

void cme_default_options(cme_options* opt)
{
    if (!opt)
        return;
    std::memset(opt, 0, sizeof *opt);
    opt->precision = CME_FP64;
    opt->integrator = CME_RK4IP;
}

const char* cme_last_error(void) { return g_err.c_str(); }
const char* cme_version(void) { return "cme-gb300 0.1 (sm_103a)"; }
long cme_kernel_launches(void) { return g_launches.load(); }

int cme_set_allocator(cme_alloc_fn alloc, cme_free_fn release, void* ctx)
{
    if ((alloc == nullptr) != (release == nullptr))
        return fail(CME_ERR_INVALID_ARG, "cme_set_allocator: give both hooks or neither");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = alloc;
    g_free = release;
    g_alloc_ctx = ctx;
    return CME_OK;
}

int cme_create(int N, const double* kappa_mu, const double* omega_mu, double g0, double kappa_ext,
               double A_in_re, double A_in_im, double sigma, cme_instance* out)
{
    if (!out)
        return fail(CME_ERR_INVALID_ARG, "cme_create: out is NULL");
    *out = nullptr;
    if (!is_pow2(N) || N < 4 || N > (1 << 20))
        return fail(CME_ERR_UNSUPPORTED_N, "cme_create: N=%d is not a power of two in [4, 2^20]", N);
    if (!kappa_mu || !omega_mu)
        return fail(CME_ERR_INVALID_ARG, "cme_create: kappa_mu and omega_mu are required");
    for (int i = 0; i < N; ++i) {
        if (!std::isfinite(kappa_mu[i]) || kappa_mu[i] < 0 || !std::isfinite(omega_mu[i]))
            return fail(CME_ERR_INVALID_ARG, "cme_create: kappa_mu[%d] or omega_mu[%d] invalid", i, i);
    }
    if (!std::isfinite(g0) || !std::isfinite(kappa_ext) || kappa_ext < 0 || !std::isfinite(A_in_re) ||
        !std::isfinite(A_in_im) || !std::isfinite(sigma))
        return fail(CME_ERR_INVALID_ARG, "cme_create: non-finite or negative scalar parameter");
    auto* p = new cme_instance_s;
    p->N = N;
    p->kappa.assign(kappa_mu, kappa_mu + N);
    p->omega.assign(omega_mu, omega_mu + N);
    p->field.assign(2 * (size_t)N, 0.0);
    p->g0 = g0;
    p->kappa_ext = kappa_ext;
    p->ain_re = A_in_re;
    p->ain_im = A_in_im;
    p->sigma = sigma;
    *out = p;
    return CME_OK;
}

int cme_create_eq2(int N, const double* kappa_rel, const double* Omega, double f0_re,
                   double f0_im, cme_instance* out)
{
    if (!out)
        return fail(CME_ERR_INVALID_ARG, "cme_create_eq2: out is NULL");
    *out = nullptr;
    if (!is_pow2(N) || N < 4 || N > (1 << 20))
        return fail(CME_ERR_UNSUPPORTED_N, "cme_create_eq2: N=%d is not a power of two in [4, 2^20]",
                    N);
    if (!Omega)
        return fail(CME_ERR_INVALID_ARG, "cme_create_eq2: Omega is required");
    // Eq. 2 is Eq. 1 in the frame of the library with tau = tau~, kappa_mu = 2 kappa_mu/kappa_0,
    // g0 = 1, sqrt(kappa_ext) A_in = f0 and omega_mu - omega_0 - sigma = Omega_mu
    std::vector<double> kap(N), om(N);
    const double O0 = Omega[N / 2];
    for (int i = 0; i < N; ++i) {
        kap[i] = 2.0 * (kappa_rel ? kappa_rel[i] : 1.0);
        om[i] = Omega[i] - O0;
    }
    if (!std::isfinite(O0))
        return fail(CME_ERR_INVALID_ARG, "cme_create_eq2: Omega_0 is not finite");
    int rc = cme_create(N, kap.data(), om.data(), 1.0, 1.0, f0_re, f0_im, -O0, out);
    if (rc != CME_OK)
        g_err = "cme_create_eq2: " + g_err;
    return rc;
}

int cme_set_field(cme_instance inst, const double* D0)
{
    if (!inst || !D0)
        return fail(CME_ERR_INVALID_ARG, "cme_set_field: NULL argument");
    for (int i = 0; i < 2 * inst->N; ++i)
        if (!std::isfinite(D0[i]))
            return fail(CME_ERR_INVALID_ARG, "cme_set_field: non-finite value at %d", i);
    inst->field.assign(D0, D0 + 2 * (size_t)inst->N);
    return CME_OK;
}

int cme_set_modes(cme_instance inst, int M)
{
    if (!inst)
        return fail(CME_ERR_INVALID_ARG, "cme_set_modes: NULL instance");
    if (M < 1 || M > inst->N)
        return fail(CME_ERR_INVALID_ARG, "cme_set_modes: M=%d outside [1, N=%d]", M, inst->N);
    inst->M = M;
    return CME_OK;
}

int cme_set_kerr(cme_instance inst, const double* g0_mu)
{
    if (!inst)
        return fail(CME_ERR_INVALID_ARG, "cme_set_kerr: NULL instance");
    if (!g0_mu) {
        inst->g0mu.clear();
        return CME_OK;
    }
    for (int i = 0; i < inst->N; ++i)
        if (!std::isfinite(g0_mu[i]))
            return fail(CME_ERR_INVALID_ARG, "cme_set_kerr: g0_mu[%d] is not finite", i);
    inst->g0mu.assign(g0_mu, g0_mu + inst->N);
    return CME_OK;
}

void cme_destroy(cme_instance inst) { delete inst; }

void cme_batch_destroy(cme_batch b)
{
    if (!b)
        return;
    if (b->stream)
        cudaStreamSynchronize(b->stream);
    b->clear_graphs();
    for (void* p : b->g_allocs)
        dev_free(p, b->free_fn, b->free_ctx);
    for (cudaEvent_t e : b->g_ev)
        if (e)
            cudaEventDestroy(e);
    if (b->g_side)
        cudaStreamDestroy(b->g_side);
    for (cudaStream_t st : b->side)
        cudaStreamDestroy(st);
    for (cudaEvent_t e : b->ev)
        cudaEventDestroy(e);
    for (void* p : b->allocs)
        dev_free(p, b->free_fn, b->free_ctx);
    if (b->own_stream && b->stream)
        cudaStreamDestroy(b->stream);
    delete b;
}

int cme_batch_create(const cme_instance* v, int count, const cme_options* opt, void* cuda_stream,
                     cme_batch* out)
{
    if (!out)
        return fail(CME_ERR_INVALID_ARG, "cme_batch_create: out is NULL");
    *out = nullptr;
    if (!v || count <= 0)
        return fail(CME_ERR_INVALID_ARG, "cme_batch_create: need at least one instance");
    cme_options o;
    cme_default_options(&o);
    if (opt)
        o = *opt;
    if (o.precision != CME_FP64 && o.precision != CME_FP32)
        return fail(CME_ERR_INVALID_ARG, "cme_batch_create: unknown precision %d", o.precision);
    if (o.integrator != CME_RK4IP && o.integrator != CME_STRANG)
        return fail(CME_ERR_INVALID_ARG, "cme_batch_create: unknown integrator %d", o.integrator);
    if (o.steps_per_launch < 0 || o.inst_per_cta < 0 || o.radix < 0)
        return fail(CME_ERR_INVALID_ARG, "cme_batch_create: negative launch option");
    for (int i = 0; i < count; ++i)
        if (!v[i])
            return fail(CME_ERR_INVALID_ARG, "cme_batch_create: instance %d is NULL", i);

    // Order instances by N so that each N forms one contiguous launch group; keep the caller's
    // order inside a group and remember the permutation (the public order is the caller's).
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i)
        order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return v[a]->N < v[c]->N; });
    for (int i = 0; i < count; ++i)
        if (order[i] != i)
            return fail(CME_ERR_INVALID_ARG,
                        "cme_batch_create: instances must be given in non-decreasing N");

    auto* b = new cme_batch_s;
    b->count = count;
    b->opt = o;
    b->prec = o.precision == CME_FP32 ? PREC_FP32 : PREC_FP64;
    b->method = o.integrator == CME_STRANG ? METHOD_STRANG : METHOD_RK4IP;
    b->elem = b->prec == PREC_FP32 ? 8 : 16;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        b->free_fn = g_free;
        b->free_ctx = g_alloc_ctx;
    }
    b->N_h.resize(count);
    b->off_h.resize(count);
    b->sigma_h.resize(count);
    long long off = 0;
    for (int i = 0; i < count; ++i) {
        b->N_h[i] = v[i]->N;
        b->off_h[i] = off;
        b->sigma_h[i] = v[i]->sigma;
        off += v[i]->N;
    }
    b->total = off;

    // launch groups
    for (int i = 0; i < count;) {
        int j = i;
        while (j < count && v[j]->N == v[i]->N)
            ++j;
        LaunchGroup g;
        g.N = v[i]->N;
        g.logN = ilog2i(g.N);
        g.first = i;
        g.count = j - i;
        g.base = b->off_h[i];
        if (g.logN > 12) {
            g.large = true;
            g.logN1 = (g.logN + 1) / 2;
            g.logN2 = g.logN / 2;
        }
        b->groups.push_back(g);
        i = j;
    }

    if (b->groups.size() > (size_t)MAX_GROUPS) {
        cme_batch_destroy(b);
        return fail(CME_ERR_INVALID_ARG, "cme_batch_create: more than %d distinct N", MAX_GROUPS);
    }
    if (o.integrator == CME_STRANG) {
        for (int i = 0; i < count; ++i)
            if (!v[i]->g0mu.empty()) {
                cme_batch_destroy(b);
                return fail(CME_ERR_INVALID_ARG,
                            "cme_batch_create: instance %d has per-mode Kerr coefficients, which "
                            "the Strang step cannot integrate exactly (use RK4IP)", i);
            }
    }
    // host-side validation of the launch options before any CUDA call
    // (the group's fields are copied out before cme_batch_destroy frees the groups)
    for (const auto& g : b->groups) {
        const int N = g.N;
        if (g.large) {
            if (o.integrator != CME_RK4IP) {
                cme_batch_destroy(b);
                return fail(CME_ERR_INVALID_ARG,
                            "cme_batch_create: N=%d > 4096 runs RK4IP only", N);
            }
            continue;
        }
        const int R = std::min(o.radix ? o.radix : default_radix(g.logN, b->prec), N);
        if (!shape_compiled(g.logN, R) || o.persistent < 0 || o.persistent > 2 ||
            !(o.cluster == 0 || o.cluster == 1 || o.cluster == 2 || o.cluster == 4 ||
              o.cluster == 8)) {
            cme_batch_destroy(b);
            return fail(CME_ERR_INVALID_ARG,
                        "cme_batch_create: launch option (radix %d, persistent %d, cluster %d) "
                        "not available for N=%d", R, o.persistent, o.cluster, N);
        }
    }
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            cme_batch_destroy(b);
            return cuda_fail(e, "cme_batch_create: cudaStreamCreate");
        }
        b->own_stream = true;
    }

    const size_t T = (size_t)b->total;
    bool ok = true;
    auto A = [&](size_t bytes) {
        void* p = b->alloc(bytes);
        if (!p)
            ok = false;
        return p;
    };
    b->hi = A(T * b->elem);
    b->lo = b->prec == PREC_FP32 ? A(T * b->elem) : nullptr;
    b->E = A(T * b->elem);
    b->e1 = A(T * b->elem);
    b->e2 = A(T * b->elem);
    b->diag = A(T * b->elem);
    b->kappa = (double*)A(T * 8);
    b->omega = (double*)A(T * 8);
    b->mode_inst = (int*)A(T * 4);
    b->stage = (double2*)A(T * 16);
    b->sigma_d = (double*)A(count * 8);
    b->g0_d = (double*)A(count * 8);
    b->pump_d = (double2*)A(count * 16);
    b->cpump_d = (double2*)A(count * 16);
    b->cpump2_d = (double2*)A(count * 16);
    b->cphi_d = (double2*)A(count * 32);
    b->inst_N = (int*)A(count * 4);
    b->status_d = (int*)A(count * 4);
    b->phys_d = (int*)A(count * 4);
    b->inst_off = (long long*)A(count * 8);
    for (auto& g : b->groups) {
        if (!b->tw.count(g.logN))
            b->tw[g.logN] = A((size_t)g.N * b->elem);
        if (g.large) {
            if (!b->tw.count(g.logN1))
                b->tw[g.logN1] = A((size_t)(1 << g.logN1) * b->elem);
            if (!b->tw.count(g.logN2))
                b->tw[g.logN2] = A((size_t)(1 << g.logN2) * b->elem);
            g.Y = A((size_t)g.count * g.N * b->elem);
            g.Z = A((size_t)g.count * g.N * b->elem);
            g.bar = (unsigned long long*)A(sizeof(unsigned long long));
            if (!b->S_large)
                b->S_large = A(T * b->elem);
        }
    }
    b->tiles_d = (FusedTile*)A(count * sizeof(FusedTile));
    b->counter_d = (int*)A(64);
    if (!ok) {
        cme_batch_destroy(b);
        return fail(CME_ERR_OOM, "cme_batch_create: device allocation of %lld modes failed",
                    (long long)T);
    }

    // host staging of the parameters (transform order for per-mode arrays)
    std::vector<double> kap(T), om(T), g0(count);
    std::vector<int> mi(T);
    std::vector<double2> pump(count), field(T);
    for (int i = 0; i < count; ++i) {
        const int N = v[i]->N;
        const long long o0 = b->off_h[i];
        const double om0 = v[i]->omega[N / 2];
        const int l = ilog2i(N), l1 = (l + 1) / 2, l2 = l / 2;
        for (int c = 0; c < N; ++c) {
            int pm = (c + N / 2) & (N - 1);  // transform position of centred index c
            if (N > 4096)                    // four-step groups: column-major m2 N1 + m1
                pm = ((pm & ((1 << l2) - 1)) << l1) + (pm >> l2);
            kap[o0 + pm] = v[i]->kappa[c];
            om[o0 + pm] = v[i]->omega[c] - om0;
            mi[o0 + pm] = i;
            field[o0 + c] = make_double2(v[i]->field[2 * c], v[i]->field[2 * c + 1]);
        }
        g0[i] = v[i]->g0mu.empty() ? v[i]->g0 : 1.0;   // per-mode: the factors carry g0_mu
        const double sk = std::sqrt(v[i]->kappa_ext);
        b->sqk_h.push_back(sk);
        pump[i] = make_double2(sk * v[i]->ain_re, sk * v[i]->ain_im);
    }
    cudaStream_t s = b->stream;
#define CPY(dst, src, bytes)                                                                  \
    do {                                                                                      \
        cudaError_t e_ = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);          \
        if (e_ == cudaSuccess)                                                                \
            e_ = cudaStreamSynchronize(s);                                                    \
        if (e_ != cudaSuccess) {                                                              \
            cme_batch_destroy(b);                                                             \
            return cuda_fail(e_, "cme_batch_create: upload");                                 \
        }                                                                                     \
    } while (0)
    CPY(b->kappa, kap.data(), T * 8);
    CPY(b->omega, om.data(), T * 8);
    CPY(b->mode_inst, mi.data(), T * 4);
    CPY(b->sigma_d, b->sigma_h.data(), count * 8);
    CPY(b->g0_d, g0.data(), count * 8);
    CPY(b->pump_d, pump.data(), count * 16);
    CPY(b->inst_N, b->N_h.data(), count * 4);
    std::vector<int> Mh(count);
    for (int i = 0; i < count; ++i)
        Mh[i] = v[i]->M > 0 ? v[i]->M : v[i]->N;
    CPY(b->phys_d, Mh.data(), count * 4);
    for (auto& g : b->groups)
        for (int i = g.first; i < g.first + g.count; ++i)
            if (Mh[i] < g.N)
                g.masked = true;
    CPY(b->inst_off, b->off_h.data(), count * 8);
    bool any_kerr = false;
    for (int i = 0; i < count; ++i)
        any_kerr |= !v[i]->g0mu.empty();
    if (any_kerr) {
        // per-mode factors in the field layout (1 for instances without per-mode coefficients)
        b->kerr_d = b->alloc(T * (b->prec == PREC_FP32 ? 4 : 8));
        if (!b->kerr_d) {
            cme_batch_destroy(b);
            return fail(CME_ERR_OOM, "cme_batch_create: device allocation of the Kerr factors");
        }
        std::vector<double> kd(T, 1.0);
        std::vector<float> kf;
        for (int i = 0; i < count; ++i) {
            if (v[i]->g0mu.empty())
                continue;
            const int N = v[i]->N, l = ilog2i(N), l1 = (l + 1) / 2, l2 = l / 2;
            for (int c = 0; c < N; ++c) {
                int pm = (c + N / 2) & (N - 1);
                if (N > 4096)
                    pm = ((pm & ((1 << l2) - 1)) << l1) + (pm >> l2);
                kd[b->off_h[i] + pm] = v[i]->g0mu[c];
            }
        }
        for (auto& g : b->groups)
            for (int i = g.first; i < g.first + g.count; ++i)
                if (!v[i]->g0mu.empty())
                    g.kerr = true;
        if (b->prec == PREC_FP32) {
            kf.assign(kd.begin(), kd.end());
            CPY(b->kerr_d, kf.data(), T * 4);
        } else {
            CPY(b->kerr_d, kd.data(), T * 8);
        }
    }
    CPY(b->stage, field.data(), T * 16);
#undef CPY
    cudaError_t e = cudaMemsetAsync(b->status_d, 0, count * 4, s);
    for (auto& kv : b->tw) {
        if (e == cudaSuccess) {
            e = launch_twiddles(1 << kv.first, b->prec, kv.second, s);
            ++g_launches;
        }
    }
    if (e == cudaSuccess) {
        e = launch_import(b->prec, (int)T, b->mode_inst, b->inst_N, b->inst_off, b->phys_d,
                          b->stage, b->hi, b->lo, s);
        ++g_launches;
    }
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cme_batch_destroy(b);
        return cuda_fail(e, "cme_batch_create: set-up kernels");
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&b->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (b->groups.size() > 1) {
        b->side.resize(b->groups.size());
        b->ev.resize(b->groups.size() + 1);
        for (auto& st : b->side) {
            e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
            if (e != cudaSuccess)
                break;
        }
        for (auto& ev : b->ev) {
            if (e == cudaSuccess)
                e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        }
        if (e != cudaSuccess) {
            cme_batch_destroy(b);
            return cuda_fail(e, "cme_batch_create: side streams");
        }
    }
    const int rc = plan_batch(b, o);
    if (rc) {
        const std::string msg = g_err;
        cme_batch_destroy(b);
        g_err = msg;
        return rc;
    }
    *out = b;
    return CME_OK;
}

int cme_batch_info(cme_batch b, int* count, long* total_modes, int* precision, int* integrator)
{
    if (!b)
        return fail(CME_ERR_INVALID_ARG, "cme_batch_info: NULL batch");
    if (count)
        *count = b->count;
    if (total_modes)
        *total_modes = (long)b->total;
    if (precision)
        *precision = b->opt.precision;
    if (integrator)
        *integrator = b->opt.integrator;
    return CME_OK;
}

void* cme_batch_stream(cme_batch b) { return b ? (void*)b->stream : nullptr; }

int cme_batch_plan(cme_batch b, int group, int* N, int* radix, int* inst_per_cta, int* cluster,
                   int* persistent)
{
    if (!b || group < 0 || group >= (int)b->groups.size())
        return fail(CME_ERR_INVALID_ARG, "cme_batch_plan: no group %d", group);
    const auto& g = b->groups[group];
    if (N)
        *N = g.N;
    if (radix)
        *radix = g.large ? g.RL : g.R;
    if (inst_per_cta)
        *inst_per_cta = g.large ? 1 : g.G;
    if (cluster)
        *cluster = g.C;
    if (persistent)
        *persistent = g.large ? (g.grid ? 2 : 1) : b->mode;
    return CME_OK;
}

}  // extern "C"

namespace {

StepArgs group_args(cme_batch b, const LaunchGroup& g)
{
    StepArgs a{};
    a.ninst = g.count;
    a.G = g.G;
    a.base = g.base;
    a.hi = b->hi;
    a.lo = b->lo;
    a.E = b->E;
    a.e1 = b->e1;
    a.e2 = b->e2;
    a.tw = b->tw[g.logN];
    a.pump = b->pump_d + g.first;
    a.cpump = b->cpump_d + g.first;
    a.cpump2 = b->cpump2_d + g.first;
    a.g0 = b->g0_d + g.first;
    a.status = b->status_d + g.first;
    a.phys = g.masked ? b->phys_d + g.first : nullptr;   // null: no padding modes in the group
    a.kerr = g.kerr ? b->kerr_d : nullptr;               // null: g0 on every mode of the group
    a.h = b->h_cur;
    a.hf = (float)b->h_cur;
    a.hhf = (float)(0.5 * b->h_cur);
    a.h6f = (float)(b->h_cur / 6.0);
    a.a2a_fault = b->a2a_fault;
    return a;
}

cudaError_t large_steps(cme_batch b, LaunchGroup& g, long long nsteps, cudaStream_t st);

cudaError_t launch_group_step(cme_batch b, LaunchGroup& g, long long nsteps, cudaStream_t st,
                              bool single_steps = false)
{
    if (g.large)
        return large_steps(b, g, nsteps, st);
    StepArgs a = group_args(b, g);
    a.nsteps = nsteps;
    a.single_steps = single_steps;
    // Concurrent groups: the groups whose blocks take over a third of an SM's shared memory
    // anyway launch with all of it, where their blocks fit one per SM together, so that each
    // such block has an SM to itself.  Where two N = 2048 blocks shared an SM, the uneven
    // N = 256 ... 4096 x 64 batch took 633 ms instead of 584 in 3 of 8 runs; with this, 584
    // in 8 of 8.
    if (b->groups.size() > 1 && g.C == 1 && b->smem_optin > 0) {
        auto heavy = [&](const LaunchGroup& q) {
            return q.C == 1 && !q.large &&
                   group_smem_bytes((int)b->elem / 2, q.logN, q.R) * (size_t)q.G * 3 >
                       (size_t)b->smem_optin;
        };
        long long blocks = 0;
        for (const auto& q : b->groups)
            if (heavy(q))
                blocks += (q.count + q.G - 1) / q.G;
        if (heavy(g) && blocks <= b->sms)
            a.smem_min = b->smem_optin;
    }
    ++g_launches;
    if (g.C > 1)
        return b->prec == PREC_FP64 ? launch_cluster_step_fp64(b->method, g.logN, g.R, g.C, a, st)
                                    : launch_cluster_step_fp32(b->method, g.logN, g.R, g.C, a, st);
    if (b->prec == PREC_FP64)
        return b->method == METHOD_RK4IP ? launch_step_fp64_rk4ip(g.logN, g.R, a, st)
                                         : launch_step_fp64_strang(g.logN, g.R, a, st);
    return b->method == METHOD_RK4IP ? launch_step_fp32_rk4ip(g.logN, g.R, a, st)
                                     : launch_step_fp32_strang(g.logN, g.R, a, st);
}

LargeArgs large_args(cme_batch b, const LaunchGroup& g)
{
    LargeArgs a{};
    a.ninst = g.count;
    a.logN1 = g.logN1;
    a.logN2 = g.logN2;
    a.base = g.base;
    a.hi = b->hi;
    a.lo = b->lo;
    a.S = b->S_large;
    a.Y = g.Y;
    a.Z = g.Z;
    a.E = b->E;
    a.e1 = b->e1;
    a.e2 = b->e2;
    a.twN = b->tw.at(g.logN);
    a.tw1 = b->tw.at(g.logN1);
    a.tw2 = b->tw.at(g.logN2);
    a.pump = b->pump_d + g.first;
    a.g0 = b->g0_d + g.first;
    a.status = b->status_d + g.first;
    a.phys = g.masked ? b->phys_d + g.first : nullptr;   // null: no padding modes in the group
    a.kerr = g.kerr ? b->kerr_d : nullptr;
    a.h = b->h_cur;
    a.hf = (float)b->h_cur;
    a.hhf = (float)(0.5 * b->h_cur);
    a.h6f = (float)(b->h_cur / 6.0);
    return a;
}

// pdl: the kernel follows another row or column kernel of the same group in the stream and
// may start while it finishes (programmatic dependent launch; the kernels order themselves).
cudaError_t large_row(cme_batch b, const LaunchGroup& g, LargeArgs a, cudaStream_t st,
                      bool pdl = false)
{
    a.G = g.G2;
    ++g_launches;
    const long long rows = (long long)g.count << g.logN1;
    return b->prec == PREC_FP64 ? launch_large_row_fp64(g.logN2, g.RL, a, rows, st, pdl)
                                : launch_large_row_fp32(g.logN2, g.RL, a, rows, st, pdl);
}

cudaError_t large_col(cme_batch b, const LaunchGroup& g, LargeArgs a, int stage, cudaStream_t st,
                      bool pdl = false)
{
    a.G = g.G1;
    a.stage = stage;
    ++g_launches;
    const long long cols = (long long)g.count << g.logN2;
    return b->prec == PREC_FP64 ? launch_large_col_fp64(g.logN1, g.RL, a, cols, st, pdl)
                                : launch_large_col_fp32(g.logN1, g.RL, a, cols, st, pdl);
}

// One RK4IP step of a four-step group: [row, col] for each of the four stages; the last column
// pass also transforms the new field for the next step's first stage.
cudaError_t large_one_step(cme_batch b, const LaunchGroup& g, const LargeArgs& a, cudaStream_t st)
{
    for (int stage = 0; stage < 4; ++stage) {
        cudaError_t e = large_row(b, g, a, st, true);
        if (e == cudaSuccess)
            e = large_col(b, g, a, stage, st, true);
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

// nsteps RK4IP steps of a four-step group: a start column pass, then whole chunks of
// LARGE_CHUNK steps replayed from a captured graph, then the remainder launched directly.
cudaError_t large_steps(cme_batch b, LaunchGroup& g, long long nsteps, cudaStream_t st)
{
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess)
        return e;
    if (g.grid && cap == cudaStreamCaptureStatusNone) {
        // every step of the call in one kernel (its barrier counter zeroed first)
        LargeArgs a = large_args(b, g);
        a.nsteps = nsteps;
        a.bar = g.bar;
        a.bar_fault = b->a2a_fault;
        e = cudaMemsetAsync(g.bar, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess)
            return e;
        ++g_launches;
        return launch_large_grid_fp32(g.logN1, g.logN2, a, (long long)g.count << g.logN2, st);
    }
    const LargeArgs a = large_args(b, g);
    e = large_col(b, g, a, LARGE_START, st);
    if (e != cudaSuccess)
        return e;
    const long long chunks = nsteps / LARGE_CHUNK;
    long long rest = nsteps % LARGE_CHUNK;
    if (chunks > 0 && cap == cudaStreamCaptureStatusNone) {
        if (!g.chunk || g.chunk_h != b->h_cur) {
            if (g.chunk)
                cudaGraphExecDestroy(g.chunk);
            g.chunk = nullptr;
            cudaGraph_t graph;
            e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess)
                return e;
            const long before = g_launches.load();
            for (int k = 0; k < LARGE_CHUNK && e == cudaSuccess; ++k)
                e = large_one_step(b, g, a, st);
            g_launches.store(before);
            cudaError_t e2 = cudaStreamEndCapture(st, &graph);
            if (e != cudaSuccess)
                return e;
            if (e2 != cudaSuccess)
                return e2;
            e = cudaGraphInstantiate(&g.chunk, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess)
                return e;
            g.chunk_h = b->h_cur;
        }
        for (long long c = 0; c < chunks; ++c) {
            g_launches += 8 * LARGE_CHUNK;
            e = cudaGraphLaunch(g.chunk, st);
            if (e != cudaSuccess)
                return e;
        }
    } else {
        rest = nsteps;
    }
    for (long long k = 0; k < rest; ++k) {
        e = large_one_step(b, g, a, st);
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

// Dynamic shared memory of the work-list kernel: the largest tile, with every group's layout
// (exchange buffers and, where used, the shared-memory accumulators) from group_smem_bytes.
size_t fused_smem(cme_batch b)
{
    size_t m = 0;
    const int tb = b->prec == PREC_FP32 ? 4 : 8;
    for (auto& g : b->groups) {
        const int Rf = fused_radix(g.logN);
        const int Pf = g.N / Rf;
        const size_t Gf = std::max(1, FUSED_THREADS / Pf);
        m = std::max(m, Gf * group_smem_bytes(tb, g.logN, Rf));
    }
    return m;
}

cudaError_t launch_fused(cme_batch b, long long nsteps)
{
    FusedArgs fa{};
    fa.ntiles = b->ntiles;
    fa.tiles = b->tiles_d;
    fa.counter = b->counter_d;
    fa.ngroups = (int)b->groups.size();
    for (int i = 0; i < fa.ngroups; ++i) {
        const auto& g = b->groups[i];
        fa.logN[i] = g.logN;
        fa.g[i] = group_args(b, g);
        fa.g[i].nsteps = nsteps;
    }
    const size_t smem = fused_smem(b);
    if (smem > (size_t)227 * 1024)
        return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaMemsetAsync(b->counter_d, 0, sizeof(int), b->stream);
    if (e != cudaSuccess)
        return e;
    const int grid = std::max(1, std::min(b->ntiles, 2 * b->sms));
    ++g_launches;
    return b->prec == PREC_FP64 ? launch_fused_fp64(b->method, fa, grid, smem, b->stream)
                                : launch_fused_fp32(b->method, fa, grid, smem, b->stream);
}

// Enqueue the step kernels for nsteps (chunked by steps_per_launch); returns kernels launched.
cudaError_t enqueue_steps(cme_batch b, long nsteps, int* nk)
{
    const long chunk = b->opt.steps_per_launch > 0 ? b->opt.steps_per_launch : nsteps;
    int k = 0;
    for (long done = 0; done < nsteps; done += chunk) {
        const long n = std::min(chunk, nsteps - done);
        cudaError_t e = cudaSuccess;
        if (b->mode == 2) {
            e = launch_fused(b, n);
            ++k;
        } else if (b->groups.size() == 1) {
            e = launch_group_step(b, b->groups[0], n, b->stream);
            ++k;
        } else {
            // fork the groups onto side streams so that they run concurrently, then join.
            // Largest N first: its kernel is the longest, and its blocks (one instance per SM
            // at N = 4096) must not queue behind the persistent blocks of lighter groups.
            e = cudaEventRecord(b->ev[0], b->stream);
            for (size_t r = 0; e == cudaSuccess && r < b->groups.size(); ++r) {
                const size_t i = b->groups.size() - 1 - r;
                e = cudaStreamWaitEvent(b->side[i], b->ev[0], 0);
                if (e == cudaSuccess)
                    e = launch_group_step(b, b->groups[i], n, b->side[i]);
                if (e == cudaSuccess)
                    e = cudaEventRecord(b->ev[1 + i], b->side[i]);
                if (e == cudaSuccess)
                    e = cudaStreamWaitEvent(b->stream, b->ev[1 + i], 0);
                ++k;
            }
        }
        if (e != cudaSuccess)
            return e;
    }
    if (nk)
        *nk = k;
    return cudaSuccess;
}

int ensure_propagators(cme_batch b, double h)
{
    if (b->h_cur == h)
        return CME_OK;
    PropArgs p{};
    p.total = (int)b->total;
    p.mode_inst = b->mode_inst;
    p.kappa = b->kappa;
    p.omega = b->omega;
    p.sigma = b->sigma_d;
    p.pump = b->pump_d;
    p.inst_N = b->inst_N;
    p.inst_off = b->inst_off;
    p.h = h;
    p.prec = b->prec;
    p.E = b->E;
    p.e1 = b->e1;
    p.e2 = b->e2;
    p.cpump = b->cpump_d;
    p.cpump2 = b->cpump2_d;
    p.ninst = b->count;
    p.cphi = b->cphi_d;
    ++g_launches;
    CME_CUDA(launch_propagators(p, b->stream), "cme_step: propagator kernel");
    b->h_cur = h;
    return CME_OK;
}

}  // namespace

extern "C" {

int cme_step(cme_batch b, double h, long nsteps)
{
    if (!b)
        return fail(CME_ERR_INVALID_ARG, "cme_step: NULL batch");
    if (!(h > 0.0) || !std::isfinite(h))
        return fail(CME_ERR_INVALID_ARG, "cme_step: h must be positive and finite (got %g)", h);
    if (nsteps < 0)
        return fail(CME_ERR_INVALID_ARG, "cme_step: nsteps must be >= 0 (got %ld)", nsteps);
    if (nsteps == 0)
        return CME_OK;
    int rc = ensure_propagators(b, h);
    if (rc)
        return rc;
    if (b->opt.use_graph && !b->has_large()) {
        auto key = std::make_pair(h, nsteps);
        auto it = b->graphs.find(key);
        if (it == b->graphs.end()) {
            cudaGraph_t graph;
            CME_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal),
                     "cme_step: begin capture");
            int nk = 0;
            const long before = g_launches.load();
            cudaError_t e = enqueue_steps(b, nsteps, &nk);
            g_launches.store(before);  // captured launches run at replay
            cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
            if (e != cudaSuccess)
                return cuda_fail(e, "cme_step: capture");
            CME_CUDA(e2, "cme_step: end capture");
            cudaGraphExec_t exec;
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            CME_CUDA(e, "cme_step: graph instantiate");
            it = b->graphs.emplace(key, std::make_pair(exec, nk)).first;
        }
        g_launches += it->second.second;
        CME_CUDA(cudaGraphLaunch(it->second.first, b->stream), "cme_step: graph launch");
    } else {
        CME_CUDA(enqueue_steps(b, nsteps, nullptr), "cme_step: kernel launch");
    }
    b->tau += h * (double)nsteps;
    return CME_OK;
}

namespace {

std::mutex g_tune_mu;
std::map<std::string, cme_options> g_tune_cache;
bool g_tune_loaded = false;

// Key of a tuning result: device, precision, integrator, h and the multiset of N.
std::string tune_key(cme_batch b, double h)
{
    cudaDeviceProp prop;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&prop, dev);
    std::string k = prop.name;
    char buf[96];
    snprintf(buf, sizeof buf, "|p%d|m%d|h%.17g", b->prec, b->method, h);
    k += buf;
    for (auto& g : b->groups) {
        snprintf(buf, sizeof buf, "|%dx%d", g.N, g.count);
        k += buf;
    }
    return k;
}

// Optional persistence: CME_TUNE_CACHE names a text file of
// "key<TAB>radix G persistent cluster" lines.
void tune_cache_load()
{
    if (g_tune_loaded)
        return;
    g_tune_loaded = true;
    const char* path = getenv("CME_TUNE_CACHE");
    if (!path)
        return;
    FILE* f = fopen(path, "r");
    if (!f)
        return;
    char line[1024];
    while (fgets(line, sizeof line, f)) {
        char* tab = strchr(line, '\t');
        if (!tab)
            continue;
        *tab = 0;
        cme_options o;
        cme_default_options(&o);
        long spl = 0;
        const int got = sscanf(tab + 1, "%d %d %d %d %ld", &o.radix, &o.inst_per_cta,
                               &o.persistent, &o.cluster, &spl);
        if (got >= 4) {
            o.steps_per_launch = got == 5 ? spl : 0;
            g_tune_cache[line] = o;
        }
    }
    fclose(f);
}

void tune_cache_store(const std::string& key, const cme_options& o)
{
    g_tune_cache[key] = o;
    const char* path = getenv("CME_TUNE_CACHE");
    if (!path)
        return;
    FILE* f = fopen(path, "a");
    if (!f)
        return;
    fprintf(f, "%s\t%d %d %d %d %ld\n", key.c_str(), o.radix, o.inst_per_cta, o.persistent,
            o.cluster, o.steps_per_launch);
    fclose(f);
}

}  // namespace

int cme_autotune(cme_batch b, double h, long probe_steps, cme_options* plan_out)
{
    if (!b || !(h > 0.0) || !std::isfinite(h) || probe_steps <= 0)
        return fail(CME_ERR_INVALID_ARG, "cme_autotune: invalid argument");
    if (b->has_large()) {   // four-step groups have a single launch plan
        if (plan_out)
            *plan_out = b->opt;
        return CME_OK;
    }
    const std::string key = tune_key(b, h);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_cache_load();
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            cme_options o = b->opt;
            o.radix = it->second.radix;
            o.inst_per_cta = it->second.inst_per_cta;
            o.persistent = it->second.persistent;
            o.cluster = it->second.cluster;
            o.steps_per_launch = it->second.steps_per_launch;
            int rc = plan_batch(b, o);
            if (rc == CME_OK) {
                if (plan_out)
                    *plan_out = b->opt;
                return CME_OK;
            }
        }
    }
    // candidates
    std::vector<cme_options> cand;
    cme_options base = b->opt;
    base.steps_per_launch = 0;
    if (b->groups.size() == 1) {
        const auto& g = b->groups[0];
        for (int R : {2, 4, 8, 16}) {
            if (R > g.N || !shape_compiled(g.logN, R))
                continue;
            for (int G : {0, 2, 4}) {
                const int P = g.N / R;
                if (G && (P >= 64 || G * P > 256))
                    continue;
                cme_options o = base;
                o.radix = R;
                o.inst_per_cta = G;
                o.persistent = 1;
                o.cluster = 1;
                cand.push_back(o);
            }
            for (int C : {2, 4, 8}) {
                if (!cluster_shape_compiled(g.logN, R, C))
                    continue;
                cme_options o = base;
                o.radix = R;
                o.inst_per_cta = 0;
                o.persistent = 1;
                o.cluster = C;
                cand.push_back(o);
            }
        }
        cme_options o = base;   // the work-list kernel also runs single-N batches
        o.radix = 0;
        o.inst_per_cta = 0;
        o.persistent = 2;
        cand.push_back(o);
    } else {
        // the work-list kernel, then per-group kernels with each cluster size (the cluster
        // size applies to the groups that have a cluster shape)
        for (int C : {0, 1, 2, 4, 8}) {
            cme_options o = base;
            o.radix = 0;
            o.inst_per_cta = 0;
            o.persistent = C == 0 ? 2 : 1;
            o.cluster = C == 0 ? 0 : C;
            cand.push_back(o);
        }
    }
    // save the field, time each candidate from the same state, restore
    const size_t fb = (size_t)b->total * b->elem;
    void* save = dev_alloc(fb * (b->prec == PREC_FP32 ? 2 : 1));
    if (!save)
        return fail(CME_ERR_OOM, "cme_autotune: no memory for the saved field");
    cme_free_fn ffn;
    void* fctx;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        ffn = g_free;
        fctx = g_alloc_ctx;
    }
    auto restore = [&]() -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(b->hi, save, fb, cudaMemcpyDeviceToDevice, b->stream);
        if (e == cudaSuccess && b->prec == PREC_FP32)
            e = cudaMemcpyAsync(b->lo, (char*)save + fb, fb, cudaMemcpyDeviceToDevice, b->stream);
        return e;
    };
    cudaError_t e = cudaMemcpyAsync(save, b->hi, fb, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess && b->prec == PREC_FP32)
        e = cudaMemcpyAsync((char*)save + fb, b->lo, fb, cudaMemcpyDeviceToDevice, b->stream);
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess)
        e = cudaEventCreate(&t0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&t1);
    int rc = CME_OK;
    if (e == cudaSuccess)
        rc = ensure_propagators(b, h);
    float best = 1e30f;
    cme_options best_o = b->opt;
    // Launch shapes first, each running the probe in one launch; then the best shape with the
    // probe split into 4 and 16 launches (steps per launch), kept only if that is faster.
    // each candidate: a warm-up of a quarter of the probe, then the probe twice, the faster
    // counting (a single timing was seen to rank plans in the wrong order on a GPU coming out
    // of idle)
    auto time_candidate = [&](const cme_options& o) {
        if (plan_batch(b, o) != CME_OK)
            return;
        e = restore();
        if (e == cudaSuccess)
            e = enqueue_steps(b, std::max(1L, probe_steps / 4), nullptr);   // warm-up
        float cand_ms = 1e30f;
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
            e = restore();
            if (e == cudaSuccess)
                e = cudaEventRecord(t0, b->stream);
            if (e == cudaSuccess)
                e = enqueue_steps(b, probe_steps, nullptr);
            if (e == cudaSuccess)
                e = cudaEventRecord(t1, b->stream);
            if (e == cudaSuccess)
                e = cudaEventSynchronize(t1);
            float ms = 0;
            if (e == cudaSuccess)
                e = cudaEventElapsedTime(&ms, t0, t1);
            if (e == cudaSuccess)
                cand_ms = std::min(cand_ms, ms);
        }
        if (e == cudaSuccess && cand_ms < best) {
            best = cand_ms;
            best_o = b->opt;
        }
    };
    // bring the GPU out of idle with the batch's current plan before anything is timed
    if (e == cudaSuccess && rc == CME_OK)
        e = enqueue_steps(b, probe_steps, nullptr);
    for (size_t c = 0; e == cudaSuccess && rc == CME_OK && c < cand.size(); ++c)
        time_candidate(cand[c]);
    const cme_options shape = best_o;
    for (long split : {4L, 16L}) {
        if (e != cudaSuccess || rc != CME_OK || probe_steps / split < 1)
            break;
        cme_options o = shape;
        o.steps_per_launch = probe_steps / split;
        time_candidate(o);
    }
    if (e == cudaSuccess)
        e = restore();
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(b->stream);
    if (t0)
        cudaEventDestroy(t0);
    if (t1)
        cudaEventDestroy(t1);
    dev_free(save, ffn, fctx);
    if (rc != CME_OK)
        return rc;
    if (e != cudaSuccess)
        return cuda_fail(e, "cme_autotune");
    rc = plan_batch(b, best_o);
    if (rc != CME_OK)
        return rc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_cache_store(key, b->opt);
    }
    if (plan_out)
        *plan_out = b->opt;
    return CME_OK;
}

int cme_synchronize(cme_batch b)
{
    if (!b)
        return fail(CME_ERR_INVALID_ARG, "cme_synchronize: NULL batch");
    CME_CUDA(cudaStreamSynchronize(b->stream), "cme_synchronize");
    std::vector<int> st(b->count);
    CME_CUDA(cudaMemcpy(st.data(), b->status_d, b->count * 4, cudaMemcpyDeviceToHost),
             "cme_synchronize: status");
    for (int i = 0; i < b->count; ++i)
        if (st[i] == 2)
            return fail(CME_ERR_TIMEOUT, "instance %d: a bounded device wait gave up", i);
    for (int i = 0; i < b->count; ++i)
        if (st[i])
            return fail(CME_ERR_NONFINITE, "instance %d has a non-finite field value", i);
    return CME_OK;
}

int cme_debug_fault(cme_batch b, int what)
{
    if (!b || what < 0 || what > 1)
        return fail(CME_ERR_INVALID_ARG, "cme_debug_fault: invalid argument");
    if (b->opt.use_graph)
        return fail(CME_ERR_INVALID_ARG,
                    "cme_debug_fault: not with use_graph (graphs keep their arguments)");
    b->a2a_fault = what;
    return CME_OK;
}

int cme_status(cme_batch b, int* per_instance)
{
    if (!b || !per_instance)
        return fail(CME_ERR_INVALID_ARG, "cme_status: NULL argument");
    CME_CUDA(cudaStreamSynchronize(b->stream), "cme_status");
    CME_CUDA(cudaMemcpy(per_instance, b->status_d, b->count * 4, cudaMemcpyDeviceToHost),
             "cme_status: copy");
    return CME_OK;
}

int cme_get_time(cme_batch b, double* tau)
{
    if (!b || !tau)
        return fail(CME_ERR_INVALID_ARG, "cme_get_time: NULL argument");
    *tau = b->tau;
    return CME_OK;
}

int cme_set_time(cme_batch b, double tau)
{
    if (!b || !std::isfinite(tau))
        return fail(CME_ERR_INVALID_ARG, "cme_set_time: invalid argument");
    b->tau = tau;
    return CME_OK;
}

int cme_get_state(cme_batch b, double* buf, int where)
{
    if (!b || !buf || (where != CME_HOST && where != CME_DEVICE))
        return fail(CME_ERR_INVALID_ARG, "cme_get_state: invalid argument");
    double2* dst = where == CME_DEVICE ? (double2*)buf : b->stage;
    ++g_launches;
    CME_CUDA(launch_export(b->prec, (int)b->total, b->mode_inst, b->inst_N, b->inst_off, b->hi,
                           b->lo, dst, 1, b->omega, b->sigma_d, b->tau, b->stream),
             "cme_get_state: export");
    if (where == CME_HOST) {
        CME_CUDA(cudaMemcpyAsync(buf, b->stage, b->total * 16, cudaMemcpyDeviceToHost, b->stream),
                 "cme_get_state: copy");
        CME_CUDA(cudaStreamSynchronize(b->stream), "cme_get_state: sync");
    }
    return CME_OK;
}

int cme_set_state(cme_batch b, const double* buf, int where)
{
    if (!b || !buf || (where != CME_HOST && where != CME_DEVICE))
        return fail(CME_ERR_INVALID_ARG, "cme_set_state: invalid argument");
    const double2* src = (const double2*)buf;
    if (where == CME_HOST) {
        CME_CUDA(cudaMemcpyAsync(b->stage, buf, b->total * 16, cudaMemcpyHostToDevice, b->stream),
                 "cme_set_state: copy");
        src = b->stage;
    }
    ++g_launches;
    CME_CUDA(launch_import(b->prec, (int)b->total, b->mode_inst, b->inst_N, b->inst_off,
                           b->phys_d, src, b->hi, b->lo, b->stream),
             "cme_set_state: import");
    CME_CUDA(cudaMemsetAsync(b->status_d, 0, b->count * 4, b->stream), "cme_set_state: status");
    if (where == CME_HOST)
        CME_CUDA(cudaStreamSynchronize(b->stream), "cme_set_state: sync");
    return CME_OK;
}

int cme_spectrum(cme_batch b, int idx, int what, double* out)
{
    if (!b || !out || idx < -1 || idx >= b->count ||
        (what != CME_POWER && what != CME_FIELD_D && what != CME_FIELD_EQ1))
        return fail(CME_ERR_INVALID_ARG, "cme_spectrum: invalid argument");
    ++g_launches;
    CME_CUDA(launch_export(b->prec, (int)b->total, b->mode_inst, b->inst_N, b->inst_off, b->hi,
                           b->lo, b->stage, what, b->omega, b->sigma_d, b->tau, b->stream),
             "cme_spectrum: export");
    const size_t per = what == CME_POWER ? 8 : 16;
    const long long first = idx < 0 ? 0 : b->off_h[idx];
    const long long n = idx < 0 ? b->total : b->N_h[idx];
    CME_CUDA(cudaMemcpyAsync(out, (char*)b->stage + first * per, n * per, cudaMemcpyDeviceToHost,
                             b->stream),
             "cme_spectrum: copy");
    CME_CUDA(cudaStreamSynchronize(b->stream), "cme_spectrum: sync");
    return CME_OK;
}

int cme_checkpoint_size(cme_batch b, size_t* bytes)
{
    if (!b || !bytes)
        return fail(CME_ERR_INVALID_ARG, "cme_checkpoint_size: NULL argument");
    *bytes = sizeof(double) + (size_t)b->total * b->elem * (b->prec == PREC_FP32 ? 2 : 1);
    return CME_OK;
}

int cme_checkpoint_save(cme_batch b, void* host_buf, size_t bytes)
{
    size_t need = 0;
    if (!b || !host_buf || cme_checkpoint_size(b, &need) || bytes < need)
        return fail(CME_ERR_INVALID_ARG, "cme_checkpoint_save: buffer too small or NULL");
    char* p = (char*)host_buf;
    std::memcpy(p, &b->tau, sizeof(double));
    const size_t fb = (size_t)b->total * b->elem;
    CME_CUDA(cudaMemcpyAsync(p + sizeof(double), b->hi, fb, cudaMemcpyDeviceToHost, b->stream),
             "cme_checkpoint_save: copy");
    if (b->prec == PREC_FP32)
        CME_CUDA(cudaMemcpyAsync(p + sizeof(double) + fb, b->lo, fb, cudaMemcpyDeviceToHost, b->stream),
                 "cme_checkpoint_save: copy");
    CME_CUDA(cudaStreamSynchronize(b->stream), "cme_checkpoint_save: sync");
    return CME_OK;
}

int cme_checkpoint_load(cme_batch b, const void* host_buf, size_t bytes)
{
    size_t need = 0;
    if (!b || !host_buf || cme_checkpoint_size(b, &need) || bytes < need)
        return fail(CME_ERR_INVALID_ARG, "cme_checkpoint_load: buffer too small or NULL");
    const char* p = (const char*)host_buf;
    double tau;
    std::memcpy(&tau, p, sizeof(double));
    const size_t fb = (size_t)b->total * b->elem;
    CME_CUDA(cudaMemcpyAsync(b->hi, p + sizeof(double), fb, cudaMemcpyHostToDevice, b->stream),
             "cme_checkpoint_load: copy");
    if (b->prec == PREC_FP32)
        CME_CUDA(cudaMemcpyAsync(b->lo, p + sizeof(double) + fb, fb, cudaMemcpyHostToDevice, b->stream),
                 "cme_checkpoint_load: copy");
    CME_CUDA(cudaMemsetAsync(b->status_d, 0, b->count * 4, b->stream), "cme_checkpoint_load: status");
    CME_CUDA(cudaStreamSynchronize(b->stream), "cme_checkpoint_load: sync");
    b->tau = tau;
    return CME_OK;
}

}  // extern "C"

namespace {

int run_diag(cme_batch b, int mode, double* out, int where, int reorder_centred, const char* who)
{
    if (!b || !out || (where != CME_HOST && where != CME_DEVICE))
        return fail(CME_ERR_INVALID_ARG, "%s: invalid argument", who);
    for (auto& g : b->groups) {
        if (g.large) {
            if (mode == DIAG_DFT)
                return fail(CME_ERR_INVALID_ARG, "%s: sign -1 is not available for N > 4096", who);
            LargeArgs la = large_args(b, g);
            la.diag_out = b->diag;
            cudaError_t e = large_col(b, g, la, LARGE_START, b->stream);
            if (e == cudaSuccess && mode == DIAG_IDFT) {
                la.diag = LDIAG_IDFT;
                e = large_row(b, g, la, b->stream);
            } else if (e == cudaSuccess) {
                e = large_row(b, g, la, b->stream);
                la.diag = LDIAG_RHS;
                if (e == cudaSuccess)
                    e = large_col(b, g, la, 0, b->stream);
            }
            if (e != cudaSuccess)
                return cuda_fail(e, who);
            continue;
        }
        StepArgs a = group_args(b, g);
        a.diag_mode = mode;
        a.diag_out = b->diag;
        ++g_launches;
        cudaError_t e = b->prec == PREC_FP64 ? launch_diag_fp64(g.logN, g.R, a, b->stream)
                                             : launch_diag_fp32(g.logN, g.R, a, b->stream);
        if (e != cudaSuccess)
            return cuda_fail(e, who);
    }
    double2* dst = where == CME_DEVICE ? (double2*)out : b->stage;
    ++g_launches;
    CME_CUDA(launch_export_plain(b->prec, (int)b->total, b->mode_inst, b->inst_N, b->inst_off,
                                 b->diag, dst, reorder_centred, b->stream),
             who);
    if (where == CME_HOST) {
        CME_CUDA(cudaMemcpyAsync(out, b->stage, b->total * 16, cudaMemcpyDeviceToHost, b->stream), who);
        CME_CUDA(cudaStreamSynchronize(b->stream), who);
    }
    return CME_OK;
}

}  // namespace

extern "C" {

int cme_transform(cme_batch b, int sign, double* out, int where)
{
    if (sign != 1 && sign != -1)
        return fail(CME_ERR_INVALID_ARG, "cme_transform: sign must be +1 or -1");
    return run_diag(b, sign > 0 ? DIAG_IDFT : DIAG_DFT, out, where, 0, "cme_transform");
}

int cme_eval_rhs(cme_batch b, double* out, int where)
{
    return run_diag(b, DIAG_RHS, out, where, 1, "cme_eval_rhs");
}

int cme_l2_peak(size_t bytes, double* bytes_per_s)
{
    if (!bytes_per_s || bytes < (1u << 20) || bytes > ((size_t)1 << 30))
        return fail(CME_ERR_INVALID_ARG, "cme_l2_peak: invalid argument");
    g_launches += 5;
    CME_CUDA(run_l2_peak(bytes, bytes_per_s), "cme_l2_peak");
    return CME_OK;
}

int cme_fma_peak(int precision, double* flops_per_s)
{
    if (!flops_per_s || (precision != CME_FP32 && precision != CME_FP64))
        return fail(CME_ERR_INVALID_ARG, "cme_fma_peak: invalid argument");
    g_launches += 4;
    CME_CUDA(run_fma_peak(precision == CME_FP32 ? PREC_FP32 : PREC_FP64, flops_per_s), "cme_fma_peak");
    return CME_OK;
}

}  // extern "C"

namespace {

// Gradient scratch: `S` checkpoints and `slots` segments of K steps of per-step data.
int ensure_grad_scratch(cme_batch b, long long S, long long slots, long long K)
{
    if (b->g_S >= S && b->g_K >= K && b->g_slots >= slots && !b->g_allocs.empty())
        return CME_OK;
    for (void* p : b->g_allocs)
        dev_free(p, b->free_fn, b->free_ctx);
    b->g_allocs.clear();
    const size_t T = (size_t)b->total, E = b->elem, C = (size_t)b->count;
    bool ok = true;
    auto A = [&](size_t bytes) {
        void* p = dev_alloc(bytes);
        if (p)
            b->g_allocs.push_back(p);
        else
            ok = false;
        return p;
    };
    b->g_ckpt_hi = A(S * T * E);
    b->g_ckpt_lo = b->prec == PREC_FP32 ? A(S * T * E) : nullptr;
    b->g_stages = A(slots * K * ADJ_VECS * T * E);
    b->g_dbar = A(T * E);
    b->g_gL = (double2*)A(T * 16);
    b->g_pbar = (double2*)A(C * 16);
    b->g_dD0 = (double2*)A(T * 16);
    b->g_loss = (double*)A(T * 8);   // per-mode loss terms
    b->g_red = (double*)A(C * 32);
    b->g_target = (double*)A(T * 8);
    b->g_domega = (double*)A(T * 8);
    b->g_dkappa = (double*)A(T * 8);
    if (!ok) {
        for (void* p : b->g_allocs)
            dev_free(p, b->free_fn, b->free_ctx);
        b->g_allocs.clear();
        b->g_S = b->g_K = b->g_slots = 0;
        return fail(CME_ERR_OOM,
                    "cme_grad: cannot allocate %lld checkpoints and %lld segments of %lld steps x "
                    "%lld modes", S, slots, K, (long long)T);
    }
    if (!b->g_side) {
        cudaError_t e = cudaStreamCreateWithFlags(&b->g_side, cudaStreamNonBlocking);
        for (auto& ev : b->g_ev)
            if (e == cudaSuccess)
                e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess)
            return cuda_fail(e, "cme_grad: recomputation stream");
    }
    b->g_S = S;
    b->g_K = K;
    b->g_slots = slots;
    return CME_OK;
}

}  // namespace

extern "C" int cme_set_grad_memory(cme_batch b, long long max_bytes)
{
    if (!b)
        return fail(CME_ERR_INVALID_ARG, "cme_set_grad_memory: NULL batch");
    b->grad_budget = max_bytes < 0 ? -1 : max_bytes;
    return CME_OK;
}

extern "C" int cme_grad(cme_batch b, double h, long nsteps, const double* target, double eps,
                        long segment, cme_grads* out)
{
    if (!b || !target || !out || !(h > 0.0) || !std::isfinite(h) || nsteps <= 0 || segment < 0 ||
        !(eps > 0.0))
        return fail(CME_ERR_INVALID_ARG, "cme_grad: invalid argument");
    if (b->has_large())
        return fail(CME_ERR_INVALID_ARG, "cme_grad: gradients are implemented for N <= 4096");
    const long long K = segment ? segment : (long long)std::ceil(std::sqrt((double)nsteps));
    const long long S = (nsteps + K - 1) / K;
    // Stored trajectory: when the per-step data of all S segments fit the budget
    // (cme_set_grad_memory; by default half the free device memory), the forward pass itself
    // stores them, segment by segment through the recomputation kernel, and the backward pass
    // reads them without recomputing anything.  Otherwise checkpoints every K steps, and each
    // segment is recomputed from its checkpoint on a second stream while the next one runs
    // backwards.
    const size_t slot_bytes = (size_t)K * ADJ_VECS * (size_t)b->total * b->elem;
    bool stored = false;
    if (b->grad_budget != 0) {
        size_t budget = (size_t)b->grad_budget;
        if (b->grad_budget < 0) {
            size_t fr = 0, tot = 0;
            if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
                cudaGetLastError();
                fr = 0;
            }
            // scratch this batch already holds is free for this call
            const size_t held = (size_t)b->g_slots * (size_t)b->g_K * ADJ_VECS *
                                (size_t)b->total * b->elem;
            budget = (fr + held) / 2;
        }
        stored = (size_t)S * slot_bytes <= budget;
    }
    int rc = stored ? ensure_grad_scratch(b, 2, S, K) : ensure_grad_scratch(b, S, 2, K);
    if (rc)
        return rc;
    rc = ensure_propagators(b, h);
    if (rc)
        return rc;
    const size_t fb = (size_t)b->total * b->elem;
    cudaStream_t st = b->stream;
    // Launch plan of the gradient's forward, recomputation and backward kernels, shared so
    // that the recomputation reproduces the forward states bit for bit.  FP32 takes 8 values
    // per thread: the backward kernel's live state spills at 16 (N = 4096: 47.3 against 50.4
    // us per gradient step with the forward at 16).  Unless the batch asked for a cluster
    // size, FP32 groups of N = 2048, 4096 take the largest cluster for which the
    // recomputation and the backward kernel, which run side by side, both get their own SMs
    // (N = 4096 x 16: 47.2 us per gradient step on one block, 28.5 on 4-block clusters,
    // 46.2 on 8-block clusters sharing SMs).  FP64 keeps the batch's plan.
    std::vector<LaunchGroup> ag(b->groups);
    for (auto& g : ag) {
        g.chunk = nullptr;   // copies never own the chunk graphs
        if (b->prec != PREC_FP32 || g.large)
            continue;
        if (b->opt.cluster == 0 && (g.logN == 11 || g.logN == 12)) {
            // with a stored trajectory the backward kernel runs alone: the whole GPU is its
            const long long share = stored ? 1 : 2;
            g.C = 1;
            for (int c : {8, 4})
                if (cluster_shape_compiled(g.logN, 8, c) && share * g.count * c <= b->sms) {
                    g.C = c;
                    break;
                }
        }
        if (g.C == 1) {
            g.R = g.N <= 4 ? 4 : 8;
            g.G = inst_per_block(g.N, g.R, 0, g.count);
        } else {
            g.R = 8;
            g.G = 1;
        }
    }
    // One launch per group of the recomputation (ADJ_RECOMPUTE) or backward role for segment sg,
    // its per-step data in slot `slot`; the recomputation starts from checkpoint `ckpt` and,
    // where out_hi is set, leaves its final state there.
    auto run_segment = [&](int role, long long sg, long long slot, long long ckpt, void* out_hi,
                           void* out_lo, cudaStream_t str) -> cudaError_t {
        for (const auto& ga : ag) {
            AdjArgs A{};
            A.s = group_args(b, ga);
            A.nsteps = nsteps;
            A.K = K;
            A.S = S;
            A.seg = sg;
            A.total = b->total;
            A.ckpt_hi = b->g_ckpt_hi;
            A.ckpt_lo = b->g_ckpt_lo ? b->g_ckpt_lo : b->g_ckpt_hi;
            A.stages = b->g_stages;
            A.dbar = b->g_dbar;
            A.gL = b->g_gL;
            A.pbar = b->g_pbar + ga.first;
            A.method = b->method;
            A.slot = slot;
            A.ckpt_slot = ckpt;
            A.out_hi = out_hi;
            A.out_lo = out_lo ? out_lo : out_hi;
            ++g_launches;
            cudaError_t e = b->prec == PREC_FP64
                                ? launch_adjoint_fp64(role, ga.logN, ga.R, ga.C, A, str)
                                : launch_adjoint_fp32(role, ga.logN, ga.R, ga.C, A, str);
            if (e != cudaSuccess)
                return e;
        }
        return cudaSuccess;
    };
    if (stored) {
        // forward through the recomputation kernel: segment s starts from checkpoint s mod 2
        // and leaves its final state in the other one (the last in the batch's field)
        CME_CUDA(cudaMemcpyAsync(b->g_ckpt_hi, b->hi, fb, cudaMemcpyDeviceToDevice, st),
                 "cme_grad: checkpoint");
        if (b->prec == PREC_FP32)
            CME_CUDA(cudaMemcpyAsync(b->g_ckpt_lo, b->lo, fb, cudaMemcpyDeviceToDevice, st),
                     "cme_grad: checkpoint");
        for (long long sg = 0; sg < S; ++sg) {
            const long long nx = (sg + 1) & 1;
            void* oh = sg + 1 == S ? b->hi : (char*)b->g_ckpt_hi + nx * fb;
            void* ol = sg + 1 == S ? b->lo
                                   : (b->g_ckpt_lo ? (char*)b->g_ckpt_lo + nx * fb : nullptr);
            CME_CUDA(run_segment(ADJ_RECOMPUTE, sg, sg, sg & 1, oh, ol, st), "cme_grad: forward");
        }
    } else {
        // forward with checkpoints at the segment starts
        for (long long s = 0; s < S; ++s) {
            CME_CUDA(cudaMemcpyAsync((char*)b->g_ckpt_hi + s * fb, b->hi, fb,
                                     cudaMemcpyDeviceToDevice, st),
                     "cme_grad: checkpoint");
            if (b->prec == PREC_FP32)
                CME_CUDA(cudaMemcpyAsync((char*)b->g_ckpt_lo + s * fb, b->lo, fb,
                                         cudaMemcpyDeviceToDevice, st),
                         "cme_grad: checkpoint");
            const long long n = std::min(K, (long long)nsteps - s * K);
            // Strang steps one by one, as the recomputation reproduces them bit for bit
            for (auto& g : ag)
                CME_CUDA(launch_group_step(b, g, n, st, true), "cme_grad: forward");
        }
    }
    // loss and its seed
    CME_CUDA(cudaMemcpyAsync(b->g_target, target, (size_t)b->total * 8, cudaMemcpyHostToDevice, st),
             "cme_grad: target");
    ++g_launches;
    CME_CUDA(launch_loss_seed(b->prec, (int)b->total, b->mode_inst, b->inst_N, b->inst_off, b->hi,
                              b->lo, b->g_target, eps, b->g_loss, b->g_dbar, st),
             "cme_grad: seed");
    // backward: segments in reverse.  Stored trajectory: each segment reads its own slot.
    // Otherwise the recomputation of segment s (states and stage values, independent of every
    // cotangent) runs on the side stream into slot s mod 2 of the stage buffer while segment
    // s + 1 runs backwards on the batch stream from the other slot.
    CME_CUDA(cudaMemsetAsync(b->g_gL, 0, (size_t)b->total * 16, st), "cme_grad: zero");
    CME_CUDA(cudaMemsetAsync(b->g_pbar, 0, (size_t)b->count * 16, st), "cme_grad: zero");
    if (stored) {
        for (long long sg = S - 1; sg >= 0; --sg)
            CME_CUDA(run_segment(ADJ_BACKWARD, sg, sg, 0, nullptr, nullptr, st),
                     "cme_grad: adjoint kernel");
    } else {
        cudaEvent_t ev_fork = b->g_ev[0], ev_rec = b->g_ev[1],
                    ev_back[2] = {b->g_ev[2], b->g_ev[3]};
        cudaStream_t side = b->g_side;
        CME_CUDA(cudaEventRecord(ev_fork, st), "cme_grad: fork");
        CME_CUDA(cudaStreamWaitEvent(side, ev_fork, 0), "cme_grad: fork");
        CME_CUDA(run_segment(ADJ_RECOMPUTE, S - 1, (S - 1) & 1, S - 1, nullptr, nullptr, side),
                 "cme_grad: recompute");
        CME_CUDA(cudaEventRecord(ev_rec, side), "cme_grad: recompute");
        for (long long sg = S - 1; sg >= 0; --sg) {
            CME_CUDA(cudaStreamWaitEvent(st, ev_rec, 0), "cme_grad: join");
            CME_CUDA(run_segment(ADJ_BACKWARD, sg, sg & 1, sg, nullptr, nullptr, st),
                     "cme_grad: adjoint kernel");
            CME_CUDA(cudaEventRecord(ev_back[sg & 1], st), "cme_grad: backward");
            if (sg >= 1) {
                // half (sg - 1) mod 2 was last read by the backward pass of segment sg + 1
                if (sg + 1 <= S - 1)
                    CME_CUDA(cudaStreamWaitEvent(side, ev_back[(sg + 1) & 1], 0), "cme_grad: wait");
                CME_CUDA(run_segment(ADJ_RECOMPUTE, sg - 1, (sg - 1) & 1, sg - 1, nullptr, nullptr,
                                     side),
                         "cme_grad: recompute");
                CME_CUDA(cudaEventRecord(ev_rec, side), "cme_grad: recompute");
            }
        }
    }
    if (b->method == METHOD_STRANG) {
        // the pump increment of the linear half flows depends on the pump and on L_0
        ++g_launches;
        CME_CUDA(launch_strang_pump_grad(b->count, b->inst_off, b->cphi_d, b->pump_d, b->g_pbar,
                                         b->g_gL, st),
                 "cme_grad: pump cotangent");
    }
    g_launches += 2;
    CME_CUDA(launch_grad_reduce(b->count, b->inst_N, b->inst_off, b->g_gL, b->g_loss, b->g_red, st),
             "cme_grad: reduce");
    CME_CUDA(launch_grad_export(b->prec, (int)b->total, b->mode_inst, b->inst_N, b->inst_off,
                                b->g_dbar, b->g_gL, b->g_red, b->g_dD0, b->g_domega, b->g_dkappa, st),
             "cme_grad: export");
    std::vector<double> red(4 * (size_t)b->count), pb(2 * (size_t)b->count);
    CME_CUDA(cudaMemcpyAsync(red.data(), b->g_red, red.size() * 8, cudaMemcpyDeviceToHost, st),
             "cme_grad: copy");
    CME_CUDA(cudaMemcpyAsync(pb.data(), b->g_pbar, pb.size() * 8, cudaMemcpyDeviceToHost, st),
             "cme_grad: copy");
    if (out->d_D0)
        CME_CUDA(cudaMemcpyAsync(out->d_D0, b->g_dD0, (size_t)b->total * 16, cudaMemcpyDeviceToHost, st),
                 "cme_grad: copy");
    if (out->d_omega)
        CME_CUDA(cudaMemcpyAsync(out->d_omega, b->g_domega, (size_t)b->total * 8,
                                 cudaMemcpyDeviceToHost, st),
                 "cme_grad: copy");
    if (out->d_kappa)
        CME_CUDA(cudaMemcpyAsync(out->d_kappa, b->g_dkappa, (size_t)b->total * 8,
                                 cudaMemcpyDeviceToHost, st),
                 "cme_grad: copy");
    CME_CUDA(cudaStreamSynchronize(st), "cme_grad: sync");
    for (int i = 0; i < b->count; ++i) {
        if (out->loss)
            out->loss[i] = red[4 * i + 3];
        if (out->d_sigma)
            out->d_sigma[i] = -red[4 * i];
        if (out->d_D2)
            out->d_D2[i] = red[4 * i + 1];
        if (out->d_D3)
            out->d_D3[i] = red[4 * i + 2];
        if (out->d_A_in) {
            out->d_A_in[2 * i] = b->sqk_h[i] * pb[2 * i];
            out->d_A_in[2 * i + 1] = b->sqk_h[i] * pb[2 * i + 1];
        }
    }
    out->stored = stored ? 1 : 0;
    b->tau += h * (double)nsteps;
    {
        std::vector<int> sw(b->count);
        CME_CUDA(cudaMemcpy(sw.data(), b->status_d, b->count * 4, cudaMemcpyDeviceToHost),
                 "cme_grad: status");
        for (int i = 0; i < b->count; ++i)
            if (sw[i] == 2)
                return fail(CME_ERR_TIMEOUT, "cme_grad: a bounded device wait gave up (instance %d)",
                            i);
    }
    return CME_OK;
}
