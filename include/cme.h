/*
 * cme.h -- C ABI of a GB300 integrator for the coupled mode equations (CMEs) of Kerr
 * frequency-comb generation, in the FFT form of Hansson, Modotto and Wabnitz
 * ("On the numerical simulation of Kerr frequency combs using coupled mode equations").
 *
 * Model (Sec. 2, Eq. 1).  For modes mu = -N/2 .. N/2-1,
 *   dA_mu/dtau = -kappa_mu/2 A_mu + delta_{mu,0} sqrt(kappa_ext) A_in e^{i sigma tau}
 *                + i g0 sum_{alpha-beta+gamma=mu} A_alpha A*_beta A_gamma
 *                       e^{i(omega_alpha - omega_beta + omega_gamma - omega_mu) tau}.
 * The library integrates it in the frame D_mu = A_mu e^{i(omega_mu - omega_0 - sigma) tau},
 * where it is autonomous:
 *   dD_mu/dtau = L_mu D_mu + delta_{mu,0} sqrt(kappa_ext) A_in + i g0 FWM_mu(D),
 *   L_mu = -kappa_mu/2 + i(omega_mu - omega_0 - sigma).
 * The four-wave-mixing (FWM) sum runs over alpha - beta + gamma = mu modulo N (the sum that
 * Eq. 4 evaluates with an N-point transform) and is computed as in Eq. 4: an inverse
 * transform over the mode number, |a|^2 a pointwise, a forward transform.
 *
 * Conventions of every entry point:
 *   - Return value: CME_OK (0) or a negative CME_ERR_* code; cme_last_error() then holds a
 *     message for the calling thread.  No entry point aborts the process.
 *   - Host arrays passed in are copied; the caller keeps ownership of everything it passes.
 *   - Complex arrays are interleaved (re, im) doubles; modes in centred order: array index
 *     i <-> mu = i - N/2 (the pumped mode mu = 0 at i = N/2).
 *   - A batch owns its device memory (allocated through cme_set_allocator's callbacks, else
 *     cudaMalloc) and runs on one CUDA stream; calls on one batch are not thread-safe.
 *   - Work is asynchronous on the batch's stream unless the entry point says it synchronises.
 */
#ifndef CME_H
#define CME_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------- */
#define CME_OK 0
#define CME_ERR_INVALID_ARG (-1)   /* null pointer, bad count, h or nsteps out of range */
#define CME_ERR_UNSUPPORTED_N (-2) /* N not a power of two in [4, 2^20] */
#define CME_ERR_CUDA (-3)          /* a CUDA runtime call failed; message has the CUDA error */
#define CME_ERR_NONFINITE (-4)     /* a field value became NaN or Inf (see cme_status) */
#define CME_ERR_TIMEOUT (-5)       /* a bounded device-side wait gave up */
#define CME_ERR_OOM (-6)           /* device allocation failed */
#define CME_ERR_STATE (-7)         /* call out of order (e.g. instance without a field) */

/* ---- options ----------------------------------------------------------------------- */
#define CME_FP64 0 /* FP64 field, transforms, Kerr term and propagators */
#define CME_FP32 1 /* FP32 field, transforms and Kerr term; propagators computed in FP64 and
                      applied as small increments; state kept as a compensated FP32 pair */

#define CME_RK4IP 0  /* fourth-order Runge-Kutta in the interaction picture (Sec. 2) */
#define CME_STRANG 1 /* Strang split step: exact linear half steps around an exact Kerr step */

#define CME_POWER 0     /* |D_mu|^2: N doubles per instance */
#define CME_FIELD_D 1   /* rotating-frame field D_mu: 2N doubles per instance */
#define CME_FIELD_EQ1 2 /* Eq. 1 frame A_mu = D_mu e^{-i(omega_mu-omega_0-sigma) tau}: 2N doubles */

#define CME_HOST 0   /* pointer argument is host memory */
#define CME_DEVICE 1 /* pointer argument is device memory on the batch's device */

typedef struct cme_instance_s* cme_instance;
typedef struct cme_batch_s* cme_batch;

typedef struct cme_options {
    int precision;         /* CME_FP64 or CME_FP32 */
    int integrator;        /* CME_RK4IP or CME_STRANG */
    int radix;             /* field elements per thread (4, 8 or 16; 2 at N = 64, 128);
                              0 = library choice.
                              For N > 4096, 4 selects the row and column kernels at 4 values
                              per thread where compiled (N1, N2 in 2^8 ... 2^10), else 8 */
    int inst_per_cta;      /* instances sharing one thread block; 0 = library choice */
    long steps_per_launch; /* steps per kernel launch; 0 = all steps of a call in one launch */
    int use_graph;         /* 1 = cme_step replays a cached CUDA graph per (h, nsteps) */
    int persistent;        /* batches with several N: 0 = library choice (1), 1 = one kernel
                              per N group (concurrent streams), 2 = one persistent work-list
                              kernel for all groups.  FP32 groups of N > 4096 (8 values per
                              thread, N = 2^15 ... 2^18): 2 runs every step of a call in one
                              kernel whose blocks meet at grid-wide barriers (cooperative
                              launch, where all its blocks fit on the GPU at once; otherwise,
                              and with 0 or 1, two kernels per RK stage) */
    int cluster;           /* thread blocks per instance (1, 2, 4 or 8) for N = 2048 and 4096
                              at 8 values per thread: C > 1 spreads each instance over a
                              thread-block cluster that runs a four-step transform (an
                              N/C-point transform inside each block, one all-to-all through
                              distributed shared memory, C-point transforms in registers;
                              one kernel per N group; also used by cme_grad).  With radix 0,
                              a cluster request selects the clusters' 8 values per thread.
                              0 = library choice: clusters only where one block per
                              instance would leave SMs idle (the batch's one-block plan uses
                              at most 2/3 of them) and not with persistent = 2; a group of
                              N = 2048 or 4096 then takes the largest C whose blocks, with
                              the other groups', stay within ~3.4 per SM: C = 8 in FP32
                              (smaller FP32 clusters do not repay their all-to-all), C = 8,
                              4 or 2 in FP64.  FP32 gradients take the largest C in {8, 4}
                              with 2 * instances * C <= SMs, since their recomputation and
                              backward kernels run side by side.  Groups without a compiled
                              cluster shape run C = 1. */
} cme_options;

/* Fill *opt with the defaults: CME_FP64, CME_RK4IP, library-chosen launch shape, no graph. */
void cme_default_options(cme_options* opt);

/* ---- instances (host-side parameter sets) -------------------------------------------- */

/* Create one CME problem (Eq. 1 parameters, Sec. 2).
 *   N          number of modes, power of two in [4, 2^20]; N <= 4096 runs one instance per
 *              thread group with the field on chip, larger N (RK4IP only, no cme_grad) runs
 *              the four-step split N = N1 N2 through row and column kernels;
 *   kappa_mu   N total losses (centred order), each >= 0;
 *   omega_mu   N cold-cavity resonance frequencies (centred order); only differences to
 *              omega_0 enter the model;
 *   g0         Kerr coefficient; kappa_ext coupling loss (>= 0);
 *   A_in       complex pump amplitude on mu = 0; sigma = omega_in - omega_0 the detuning.
 * The initial field is zero until cme_set_field.  Errors: INVALID_ARG, UNSUPPORTED_N. */
int cme_create(int N, const double* kappa_mu, const double* omega_mu, double g0,
               double kappa_ext, double A_in_re, double A_in_im, double sigma,
               cme_instance* out);

/* Create an instance of the normalised Eq. 2 (Sec. 2):
 *   dA~_mu/dtau~ = (-kappa_mu/kappa_0 + i Omega_mu) A~_mu + delta_{mu,0} f0
 *                  + i sum_{alpha-beta+gamma=mu} A~_alpha A~*_beta A~_gamma,
 * whose time is tau~ = kappa_0 tau / 2: h, nsteps and the accumulated time of cme_step are then
 * in units of tau~, and the field is A~ (in the frame of Omega_mu, like D of cme_create).
 *   kappa_rel  N values kappa_mu / kappa_0 (centred), each >= 0; NULL: all 1;
 *   Omega      N normalised detunings Omega_mu (centred; Omega_0 is the pump detuning term);
 *   f0         complex normalised pump.
 * Equivalent to cme_create with kappa_mu = 2 kappa_rel, omega_mu = Omega_mu - Omega_0, g0 = 1,
 * kappa_ext = 1, A_in = f0, sigma = -Omega_0.  Errors as cme_create. */
int cme_create_eq2(int N, const double* kappa_rel, const double* Omega, double f0_re,
                   double f0_im, cme_instance* out);

/* Set the initial rotating-frame field D_mu(0): 2N doubles, interleaved, centred order. */
int cme_set_field(cme_instance inst, const double* D0);

/* Number of physical modes M (1 <= M <= N; default N): the zero padding of Sec. 2, where 201
 * modes run in a 256-point transform.  Of the N modes only the centred M,
 * mu = -floor(M/2) .. M - floor(M/2) - 1, are physical.  The others are padding: they start
 * at zero (whatever the field set for them) and stay there, and the four-wave-mixing sum runs
 * over physical modes only and has no term on padding modes.  With N >= 2M no index triple wraps
 * around into the physical band, and the sum is the linear (non-circular) sum of the M-mode
 * system; M < N < 2M is the paper's own padding, where some triples still wrap.  The kappa,
 * omega and field arrays keep N entries; padding entries are ignored.  Errors: INVALID_ARG. */
int cme_set_modes(cme_instance inst, int M);

/* Per-mode Kerr coefficients g0_mu (N values, centred, finite), or NULL to go back to g0 on
 * every mode.  Sec. 2 notes that a constant g0 is no necessary restriction and that the
 * coupled mode equations take frequency-dependent coefficients easily; the form implemented
 * is the coefficient of the output mode,
 *   dD_mu/dtau = L_mu D_mu + delta_{mu,0} sqrt(kappa_ext) A_in + i g0_mu FWM_mu(D),
 * which keeps Eq. 4: a per-mode factor after the forward transform.  (A coefficient that
 * depends on the whole quadruplet alpha, beta, gamma, mu has no transform form.)  RK4IP only:
 * a batch with such an instance and the Strang integrator is refused, because the split step's
 * exact Kerr flow needs one coefficient for all modes.  Errors: INVALID_ARG. */
int cme_set_kerr(cme_instance inst, const double* g0_mu);

void cme_destroy(cme_instance inst);

/* ---- batches (device-resident sets of instances) --------------------------------------- */

/* Build a batch from `count` instances (copied; the instances may be destroyed afterwards),
 * given in non-decreasing N.  Instances may differ in N; each distinct N forms its own launch
 * group.  `cuda_stream` is a
 * cudaStream_t; NULL makes the batch create and own a non-blocking stream.  The field starts
 * at the instances' initial fields, tau = 0.  Errors: INVALID_ARG, UNSUPPORTED_N, CUDA, OOM. */
int cme_batch_create(const cme_instance* v, int count, const cme_options* opt,
                     void* cuda_stream, cme_batch* out);

void cme_batch_destroy(cme_batch b);

/* count = instances; total_modes = sum of N; fills any non-null pointer. */
int cme_batch_info(cme_batch b, int* count, long* total_modes, int* precision, int* integrator);

/* The batch's stream (cudaStream_t). */
void* cme_batch_stream(cme_batch b);

/* The launch plan the library chose for launch group `group` (0-based, groups in increasing N):
 * N, values per thread, instances per block, blocks per instance (cluster) and the batch's
 * persistent mode (1 or 2; for N > 4096 groups 2 means the grid-barrier kernel, 1 the kernel
 * sequence).  Any output pointer may be NULL.  Errors: INVALID_ARG. */
int cme_batch_plan(cme_batch b, int group, int* N, int* radix, int* inst_per_cta, int* cluster,
                   int* persistent);

/* Advance every instance by nsteps steps of size h (> 0) of the batch's integrator (Sec. 2:
 * RK4 or split step, with the FWM term evaluated through Eq. 4).  Asynchronous.  The first
 * call with a new h also recomputes the per-mode propagators exp(L h/2), expm1(L h/2),
 * expm1(L h) in FP64.  Strang: within one launch the linear half flow that closes a step and
 * the one that opens the next are applied as their exact composition over h, so n steps cost
 * n + 1 linear flows; the result is that of n single steps up to rounding.  nsteps = 0 is a
 * no-op.  Errors: INVALID_ARG, CUDA. */
int cme_step(cme_batch b, double h, long nsteps);

/* Pick the fastest launch plan for this batch and step size h by timing `probe_steps` steps of
 * each candidate (values per thread, instances per block, blocks per instance, per-group vs
 * persistent launch) on the device, each as one launch; then the best of them with the probe
 * split into 4 and into 16 launches (steps_per_launch = probe_steps / 4, / 16), kept only where
 * that is faster.  The field is saved before and restored after, so the batch state is unchanged.
 * The chosen plan replaces the batch's options for later cme_step calls; *plan_out (may be
 * NULL) receives it.  Synchronises.  Errors: INVALID_ARG, CUDA. */
int cme_autotune(cme_batch b, double h, long probe_steps, cme_options* plan_out);

/* Wait for the batch's stream; returns CME_ERR_TIMEOUT if any instance's status is 2, else
 * CME_ERR_NONFINITE if any instance's status is set. */
int cme_synchronize(cme_batch b);

/* Copy out one instance (idx >= 0) or all instances concatenated (idx = -1) to host memory:
 * what = CME_POWER, CME_FIELD_D or CME_FIELD_EQ1.  Synchronises. */
int cme_spectrum(cme_batch b, int idx, int what, double* out);

/* Whole-batch field, FP64 interleaved centred rotating frame, all instances concatenated
 * (2 * total_modes doubles).  `where` = CME_HOST (synchronises) or CME_DEVICE (asynchronous;
 * `buf` must be 8-byte aligned device memory).  cme_set_state also clears the status words.
 * In CME_FP32 batches the FP64 value is split into the compensated (hi, lo) pair. */
int cme_get_state(cme_batch b, double* buf, int where);
int cme_set_state(cme_batch b, const double* buf, int where);

/* Bit-exact checkpoint of the internal state (field words plus tau): size in bytes, then
 * copy out / in through host memory.  Synchronises. */
int cme_checkpoint_size(cme_batch b, size_t* bytes);
int cme_checkpoint_save(cme_batch b, void* host_buf, size_t bytes);
int cme_checkpoint_load(cme_batch b, const void* host_buf, size_t bytes);

/* Accumulated time tau (FP64 sum of h * nsteps over cme_step calls). */
int cme_get_time(cme_batch b, double* tau);
int cme_set_time(cme_batch b, double tau);

/* Per-instance status words (host array of `count` ints): 0 = finite, 1 = non-finite value
 * seen at the end of a launch, 2 = a bounded wait of a cluster all-to-all or of a grid
 * barrier (persistent = 2 for N > 4096) gave up (the instance's results are not valid).
 * Synchronises. */
int cme_status(cme_batch b, int* per_instance);

/* Test of the failure path of the bounded device waits (not for normal use): what = 1 makes
 * the cluster all-to-alls of later cme_step / cme_grad calls expect 8 bytes more than are
 * sent, and the grid barriers of the N > 4096 grid kernel one arrival more than there are
 * blocks, and both poll only briefly, so their waits run out; the instances then report status 2 and
 * cme_synchronize / cme_grad return CME_ERR_TIMEOUT, with no device fault.  what = 0 restores
 * normal operation (cme_set_state clears the status words).  Batches without use_graph only.
 * Errors: INVALID_ARG. */
int cme_debug_fault(cme_batch b, int what);

/* ---- gradients (discrete adjoint) ------------------------------------------------------- */

/* Gradients of the log-power-spectrum misfit at the final step, per instance
 *     L = sum_mu (log10(|D_mu|^2 + eps) - T_mu)^2 ,
 * through nsteps steps of size h of the batch's integrator (Sec. 2: the RK4 method, RK4IP here,
 * or the split-step Fourier method, the Strang split step here).  Every pointer is a host array
 * and may be NULL to skip that output; complex cotangents are dL/dRe + i dL/dIm, interleaved;
 * per-mode arrays are centred. */
typedef struct cme_grads {
    double* loss;    /* [count] L of each instance */
    double* d_sigma; /* [count] dL/dsigma */
    double* d_A_in;  /* [2*count] dL/dRe A_in + i dL/dIm A_in */
    double* d_D2;    /* [count] sum_mu dL/domega_mu mu^2/2 (omega_mu = D2 mu^2/2 + D3 mu^3/6) */
    double* d_D3;    /* [count] sum_mu dL/domega_mu mu^3/6 */
    double* d_omega; /* [total_modes] dL/domega_mu */
    double* d_kappa; /* [total_modes] dL/dkappa_mu */
    double* d_D0;    /* [2*total_modes] cotangent of the field at the start of the call */
    int stored;      /* out: 1 if the call stored the whole trajectory, 0 if it checkpointed and
                        recomputed segments (see cme_grad) */
} cme_grads;

/* Run nsteps steps of the batch's integrator from the current field in segments of `segment`
 * steps (0 = ceil(sqrt(nsteps))), evaluate L against the target T (total_modes doubles: log10
 * powers, centred, host memory), then run the discrete adjoint backwards over the segments.
 * Two schedules:
 *   - stored trajectory, where the per-step data of the whole run fit the budget of
 *     cme_set_grad_memory (by default half the device memory free at the call): the forward
 *     pass stores them as it goes, and the backward pass reads them back; nothing is
 *     recomputed (N = 4096 x 16 instances, 10000 FP32 steps: 42 GB, FP64: 84 GB);
 *   - otherwise checkpoints at the segment starts; each segment is recomputed from its
 *     checkpoint, the recomputation of the next segment overlapping the backward pass of the
 *     current one on a second stream (sqrt(nsteps) checkpointing).
 * Both give the same gradient to rounding (the launch plans may differ: the stored schedule's
 * backward kernel has the GPU to itself).  RK4IP: per step the state, the
 * three stage values and the time-domain fields of the four stage inputs are recomputed, and
 * the backward pass runs four vector-Jacobian products of the right-hand side.  Strang: the
 * state, the time-domain field of the Kerr flow and the state after it are recomputed, and the
 * backward pass runs the exact Kerr flow's vector-Jacobian product (two transforms) between the
 * two linear half flows; the pump increment (exp(L_0 h/2) - 1)/L_0 sqrt(kappa_ext) A_in passes
 * its cotangent to A_in and to L_0.  The batch ends at the final field (tau advanced by
 * h nsteps).  Scratch memory -- the stored trajectory, 8 field vectors per step, or
 * ceil(nsteps/segment) checkpoints and 8 * segment field vectors per segment for two segments --
 * is allocated on the first call and kept with the batch (and reallocated when a later call
 * needs more).  N <= 4096 only.  Synchronises.  Errors: INVALID_ARG, CUDA, OOM, TIMEOUT (a
 * bounded wait of a cluster all-to-all gave up). */
int cme_grad(cme_batch b, double h, long nsteps, const double* target, double eps, long segment,
             cme_grads* out);

/* Budget in bytes for cme_grad's stored trajectory: -1 (default) = half the device memory
 * free at each call, 0 = never store (always checkpoint and recompute), > 0 = store when the
 * trajectory needs at most max_bytes.  Errors: INVALID_ARG. */
int cme_set_grad_memory(cme_batch b, long long max_bytes);

/* ---- hot-path pieces, for testing ----------------------------------------------------- */

/* Unnormalised transform over the mode number of the current field (Eq. 4), run by the same
 * device code as cme_step: sign = +1 gives a_j = sum_mu D_mu e^{+2 pi i j mu/N} for time
 * samples j = 0..N-1; sign = -1 gives sum_mu D_mu e^{-2 pi i j mu/N}.  Output 2 * total_modes
 * doubles (per instance: j-ordered samples), to host (synchronises) or device memory. */
int cme_transform(cme_batch b, int sign, double* out, int where);

/* Right-hand side F(D) = delta_{mu,0} sqrt(kappa_ext) A_in + i g0 FWM(D) of the current
 * field, FWM through Eq. 4 on the device (centred order, 2 * total_modes doubles). */
int cme_eval_rhs(cme_batch b, double* out, int where);

/* ---- integration without device allocation ------------------------------------------- */

/* Size of the device array that cme_rk4ip_noalloc uses for all of its scratch memory. */
#define CME_NOALLOC_SCRATCH_BYTES (16u << 20)

/* The paper has no counterpart to this entry point; it exists for callers that may not
 * allocate device memory themselves -- for example an application whose device memory all comes
 * from its own fixed-size pool, or code running between other asynchronous work where
 * cudaMalloc, which can synchronise the whole device, must not be called.
 *
 * Advances `count` instances of N modes (power of two in [4, 4096]) by nsteps RK4IP steps of
 * size h in FP64, in place, and calls no cudaMalloc, cudaFree or allocating library routine.
 * It runs the one-block step kernels of cme_step with the launch shape (values per thread,
 * instances per block) that cme_batch_create chooses for an FP64 RK4IP batch of these
 * instances under default options before its choice of thread-block clusters: the result is
 * bit for bit that of such a batch created with cluster = 1.  Where the default batch spreads
 * N = 2048 or 4096 instances over clusters, the two agree to rounding only.  All pointers are
 * device memory owned by the caller:
 *   d_kappa, d_omega  N * count doubles each: kappa_mu and omega_mu per instance, centred;
 *   d_inst            5 * count doubles: (g0, kappa_ext, Re A_in, Im A_in, sigma) per instance;
 *   d_field           2 * N * count doubles (in/out): rotating-frame field, interleaved, centred.
 * Work is enqueued on cuda_stream (NULL: the legacy default stream) and the call returns without
 * waiting.  Scratch: one static device array of CME_NOALLOC_SCRATCH_BYTES (16 MiB), held by
 * every GPU that loads the library until the process exits; it needs about 84 bytes per mode
 * plus 16 N, so at most about 190000 modes per call -- larger sets are rejected with
 * CME_ERR_INVALID_ARG.  Every call shares that array and it keeps the previous call's
 * contents (the status words are cleared by each call): calls that overlap on the GPU, on
 * different streams or from different threads, race and corrupt each other.  The first call on
 * a device takes the array's device address with cudaGetSymbolAddress and keeps it; make that
 * first call before any stream capture, and do not call this entry point again on a device
 * after cudaDeviceReset (the kept address belongs to the context that was reset).  Non-finite
 * results are not reported: the call returns before the kernels run and reads nothing back,
 * so a field that overflows to Inf or NaN comes back in d_field with CME_OK; check d_field.
 * Six kernels per call (five when nsteps = 0) count towards cme_kernel_launches.
 * Errors: UNSUPPORTED_N, INVALID_ARG, CUDA. */
int cme_rk4ip_noalloc(int N, int count, double h, long nsteps, const double* d_kappa,
                      const double* d_omega, const double* d_inst, double* d_field,
                      void* cuda_stream);

/* ---- library ------------------------------------------------------------------------ */

/* Device allocation hooks used by every later batch: alloc(bytes, ctx) returns device memory
 * or NULL; release(ptr, ctx) frees it.  Pass NULLs to restore cudaMalloc / cudaFree. */
typedef void* (*cme_alloc_fn)(size_t bytes, void* ctx);
typedef void (*cme_free_fn)(void* ptr, void* ctx);
int cme_set_allocator(cme_alloc_fn alloc, cme_free_fn release, void* ctx);

/* Measured throughput of dependent-free fused multiply-adds on the current device, in
 * flop/s (2 flop per FMA), for CME_FP32 or CME_FP64; runs for a few tens of ms. */
int cme_fma_peak(int precision, double* flops_per_s);

/* Measured bandwidth of copying between two buffers of together at most `bytes` (1 MiB .. 1 GiB;
 * each buffer the largest power of two of float4 that fits): read plus written bytes per
 * second, best of four launches of 32 passes after a first launch that brings both buffers
 * into the cache.  With `bytes` well under the 129 MB L2 of this GPU this is the L2 bandwidth
 * a kernel whose working set stays in L2 can reach (the large-N kernels' roof); with more, the
 * HBM bandwidth.  Allocates and frees its buffers; runs for a few ms. */
int cme_l2_peak(size_t bytes, double* bytes_per_s);

/* Number of kernels this library has launched in the calling process (for accounting). */
long cme_kernel_launches(void);

const char* cme_last_error(void);
const char* cme_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CME_H */
