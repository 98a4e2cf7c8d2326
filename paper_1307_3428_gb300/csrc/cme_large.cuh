// Large-N RK4IP (N = N1 N2 > 4096): the transforms over the mode number are split into
// N2 column transforms of length N1 and N1 row transforms of length N2 (the four-step
// factorisation of the DFT), each done by one thread group with the in-block transform code.
//
// Index maps (transform order m = mu mod N, time index j):
//     m = m1 N2 + m2,   j = j1 + N1 j2.
// Inverse transform a_j = sum_m x_m exp(+2 pi i j m / N):
//     Y[j1][m2] = exp(+2 pi i j1 m2 / N) sum_m1 x[m1 N2 + m2] exp(+2 pi i j1 m1 / N1)   (col)
//     a[j1 + N1 j2] = sum_m2 Y[j1][m2] exp(+2 pi i j2 m2 / N2)                         (row)
// Forward transform X_m = sum_j b_j exp(-2 pi i j m / N):
//     Z[j1][m2] = exp(-2 pi i j1 m2 / N) sum_j2 b[j1 + N1 j2] exp(-2 pi i j2 m2 / N2)   (row)
//     X[m1 N2 + m2] = sum_j1 Z[j1][m2] exp(-2 pi i j1 m1 / N1)                         (col)
// One RK stage is therefore two kernels:
//   row: load Y row j1, inverse over m2, Kerr term (i g0/N) |a|^2 a, forward over j2,
//        twiddle, store Z row j1 (the time-domain field never leaves registers);
//   col: load Z column m2, forward over j1, pump, Runge-Kutta combination of the stage (the
//        same increment form as the in-block kernels), inverse over m1 of the next stage's
//        input, twiddle, store Y column m2.
// The field, the accumulator S and the propagators stay in HBM (L2-resident at these sizes),
// stored column-major (mode m1 N2 + m2 at position m2 N1 + m1) so that the column kernel reads
// them contiguously; Y (column-major) and Z (row-major) are the inter-pass buffers (scratch),
// laid out so that both kernels store them contiguously and only read them strided: a kernel
// waits at its exit for its stores, and strided stores made that wait the longest stall (N =
// 2^17: 31.7 -> 29.6 us per step with the strides moved to the loads).
#pragma once

#include "cme_step.cuh"

namespace cme {

enum { LARGE_START = -1, LARGE_FINAL = 4 };
enum { LDIAG_NONE = 0, LDIAG_IDFT = 1, LDIAG_RHS = 2 };

struct LargeArgs {
    int ninst;
    int logN1, logN2;        // column transform length N1 = 2^logN1, row length N2 = 2^logN2
    int G;                   // thread groups (rows or columns) per block
    long long base;          // first mode offset of the group
    void* hi;                // field (FP32: hi part)
    void* lo;                // FP32 compensation word
    void* S;                 // Runge-Kutta accumulator
    void* Y;                 // [ninst][N2][N1] column-pass output, column-major (m2 N1 + j1)
    void* Z;                 // [ninst][N1][N2] row-pass output, row-major (j1 N2 + m2)
    const void* E;
    const void* e1;
    const void* e2;
    const void* twN;         // exp(2 pi i k / N), k < N
    const void* tw1;         // exp(2 pi i k / N1)
    const void* tw2;         // exp(2 pi i k / N2)
    const double2* pump;     // per instance (group-relative)
    const double* g0;
    int* status;
    const int* phys;         // per-instance physical mode count M (null: all N)
    const void* kerr;        // per-mode Kerr factors g0_mu / g0 (field layout), or null
    double h;
    float hf, hhf, h6f;
    int stage;               // col kernel: LARGE_START, 0..3, LARGE_FINAL
    int diag;                // LDIAG_*: write to diag_out instead of continuing
    void* diag_out;          // [ninst][N] transform order (rhs) or time order (idft)
    // grid-barrier kernel only
    long long nsteps;        // steps of the launch
    unsigned long long* bar; // arrival counter of the grid barriers, zero at launch
    int bar_fault;           // test of the bounded waits: every barrier expects one arrival more
};

// Programmatic dependent launch: the step's kernels are launched so that each may start while
// its predecessor finishes.  A kernel reads only constant data (propagators, twiddles) before
// pdl_wait(), which returns once the predecessor has completed and its writes are visible; every
// read of mutable data and every write comes after it.  pdl_trigger() after the wait lets the
// successor start its own constant prologue.  Launched without the attribute, both are no-ops.
CME_DEV void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
CME_DEV void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Row pass: instance i = row / N1, row j1 = row mod N1.
template <typename T, int LOGN2, int R>
__global__ void __launch_bounds__(max_threads<LOGN2, R>()) large_row_kernel(const LargeArgs A)
{
    using GR = Group<T, LOGN2, R>;
    constexpr int N2 = GR::N, P = GR::P;
    extern __shared__ __align__(16) unsigned char smem[];
    const int N1 = 1 << A.logN1;
    const long long N = (long long)N1 * N2;
    const int g = threadIdx.x / P;
    const long long rows = (long long)A.ninst * N1;
    long long row = (long long)blockIdx.x * A.G + g;
    const bool valid = row < rows;
    if (!valid)
        row = rows - 1;
    const int inst = (int)(row / N1);
    const int j1 = (int)(row - (long long)inst * N1);
    GR grp;
    grp.setup(smem, g, threadIdx.x - g * P, A.tw2);
    const int t = grp.t;
    const long long ibase = (long long)inst * N;   // offset of this instance in Y / Z
    // the output twiddles (constant) before the wait, so that their latency overlaps it
    cx<T> w[R];
#pragma unroll
    for (int j = 0; j < R; ++j)
        w[j] = gload<T>(A.twN, ((long long)j1 * (t + j * P)) & (N - 1));
    pdl_wait();
    pdl_trigger();
    const cx<T>* yrow = reinterpret_cast<const cx<T>*>(A.Y) + ibase + (long long)t * N1 + j1;
    cx<T> x[R];
#pragma unroll
    for (int j = 0; j < R; ++j)
        x[j] = yrow[(long long)j * P * N1];
    if (A.diag == LDIAG_IDFT) {
        grp.inverse(x, 0);
        if (valid) {
            cx<T>* d = reinterpret_cast<cx<T>*>(A.diag_out) + A.base + ibase + j1;
#pragma unroll
            for (int j = 0; j < R; ++j)
                d[(long long)(t + j * P) * N1] = x[j];   // a[j1 + N1 j2], j2 = t + jP
        }
        return;
    }
    const T gN = (T)A.g0[inst] * ((T)1 / (T)N);   // N is a power of two: exact scaling
    grp.rhs(x, gN, cx<T>{T(0), T(0)});   // forward(i g0/N |a|^2 a) over j2, natural m2
    cx<T>* zcol = reinterpret_cast<cx<T>*>(A.Z) + ibase + (long long)j1 * N2 + t;
    if (valid) {
#pragma unroll
        for (int j = 0; j < R; ++j)
            zcol[j * P] = cmulc(x[j], w[j]);   // * exp(-2 pi i j1 m2 / N)
    }
}

// Column pass: instance i = col / N2, column m2 = col mod N2.  One instantiation per stage ST
// (LARGE_START, 0 ... 3, LARGE_FINAL; A.stage is ST): each holds only its stage's code.
template <typename T, int LOGN1, int R, int ST>
__global__ void __launch_bounds__(max_threads<LOGN1, R>()) large_col_kernel(const LargeArgs A)
{
    using GR = Group<T, LOGN1, R>;
    constexpr int N1 = GR::N, P = GR::P;
    constexpr bool COMP = GR::COMP;
    extern __shared__ __align__(16) unsigned char smem[];
    const int N2 = 1 << A.logN2;
    const long long N = (long long)N1 * N2;
    const int g = threadIdx.x / P;
    const long long cols = (long long)A.ninst * N2;
    long long col = (long long)blockIdx.x * A.G + g;
    const bool valid = col < cols;
    if (!valid)
        col = cols - 1;
    const int inst = (int)(col / N2);
    const int m2 = (int)(col - (long long)inst * N2);
    GR grp;
    grp.setup(smem, g, threadIdx.x - g * P, A.tw1);
    const int t = grp.t;
    const long long ibase = (long long)inst * N;
    // element j of this thread: m1 (or j1) = t + jP, stored column-major at m2 N1 + t + jP
    const long long e0 = ibase + (long long)m2 * N1 + t;
    const long long estride = P;
    const long long f0 = A.base + e0;   // same element in the field / per-mode arrays

    cx<T>* hi = reinterpret_cast<cx<T>*>(A.hi) + f0;
    cx<T>* lo = reinterpret_cast<cx<T>*>(A.lo) + f0;
    cx<T>* Sp = reinterpret_cast<cx<T>*>(A.S) + f0;
    const cx<T>* Ep = reinterpret_cast<const cx<T>*>(A.E) + f0;
    const cx<T>* e1p = reinterpret_cast<const cx<T>*>(A.e1) + f0;
    const cx<T>* e2p = reinterpret_cast<const cx<T>*>(A.e2) + f0;
    constexpr int st = ST;
    // Every operand of the Runge-Kutta combination and the output twiddles are loaded here,
    // before the transforms, so that their latency overlaps the first transform: the constant
    // ones (propagators, twiddles) even before the wait for the preceding kernel.
    cx<T> Dh[R], Dl[R], Sv[R], Ev[R], ev[R], w[R];
    const bool rk = A.diag != LDIAG_RHS;
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const long long o = j * estride;
        Dh[j] = Dl[j] = Sv[j] = Ev[j] = ev[j] = w[j] = cx<T>{T(0), T(0)};
        if (rk) {
            if (st >= 0 && st <= 2)
                Ev[j] = gload<T>(Ep, o);
            if (st == 0 || st == 1)
                ev[j] = gload<T>(e1p, o);
            else if (st == 2 || st == 3)
                ev[j] = gload<T>(e2p, o);
            if (st != LARGE_FINAL)
                w[j] = gload<T>(A.twN, ((long long)(t + j * P) * m2) & (N - 1));
        }
    }
    pdl_wait();
    pdl_trigger();
    if (rk) {
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const long long o = j * estride;
            Dh[j] = hi[o];
            if (st >= 1 && st <= 3)
                Sv[j] = Sp[o];
            if constexpr (COMP) {
                if (st == 3)
                    Dl[j] = lo[o];
            }
        }
    }

    cx<T> x[R];
    if constexpr (ST != LARGE_START) {
        // forward transform over j1 of Z column m2, as conj(inverse(conj(.)))
        const cx<T>* z = reinterpret_cast<const cx<T>*>(A.Z) + ibase + (long long)t * N2 + m2;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const cx<T> v = z[(long long)j * P * N2];
            x[j] = {v.re, -v.im};
        }
        grp.inverse(x, 1);
#pragma unroll
        for (int j = 0; j < R; ++j)
            x[j].im = -x[j].im;
        if (A.kerr) {
            // per-mode Kerr coefficient of the output mode (the instance's g0 is then 1)
            const T* km = reinterpret_cast<const T*>(A.kerr) + f0;
#pragma unroll
            for (int j = 0; j < R; ++j)
                x[j] = cscale(x[j], __ldg(km + j * estride));
        }
        if (A.phys) {
            // padding modes (outside the centred M physical ones) get no FWM term
            const int M = A.phys[inst];
            if (M < N) {
                const long long mlo = -(M / 2), mhi = M - M / 2 - 1;
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    const long long m = (long long)(t + j * P) * N2 + m2;   // mode mu mod N
                    const long long mu = m >= N / 2 ? m - N : m;
                    if (mu < mlo || mu > mhi)
                        x[j] = cx<T>{T(0), T(0)};
                }
            }
        }
        if (t == 0 && m2 == 0) {
            const double2 pd = A.pump[inst];
            x[0] = cadd(x[0], cx<T>{(T)pd.x, (T)pd.y});
        }
        if (A.diag == LDIAG_RHS) {
            if (valid) {
                cx<T>* d = reinterpret_cast<cx<T>*>(A.diag_out) + f0;
#pragma unroll
                for (int j = 0; j < R; ++j)
                    d[j * estride] = x[j];
            }
            return;
        }
    }
    T h, hh, h6;
    if constexpr (sizeof(T) == 4) {
        h = A.hf;
        hh = A.hhf;
        h6 = A.h6f;
    } else {
        h = A.h;
        hh = 0.5 * A.h;
        h6 = A.h / 6.0;
    }
    // Runge-Kutta combination of stage st (same increment form as rk4ip_step) and the next
    // stage's input; LARGE_START only loads D, LARGE_FINAL finishes the step without going on.
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const long long o = j * estride;
        cx<T> D = Dh[j];
        if (st == LARGE_START) {
            x[j] = D;
        } else if (st == 0) {
            const cx<T> k1 = cmul(Ev[j], x[j]);
            Sp[o] = cmul(Ev[j], k1);
            x[j] = cadd(D, caxpy(cmul(ev[j], D), hh, k1));
        } else if (st == 1) {
            Sp[o] = caxpy(Sv[j], T(2), cmul(Ev[j], x[j]));
            x[j] = cadd(D, caxpy(cmul(ev[j], D), hh, x[j]));
        } else if (st == 2) {
            const cx<T> Ek3 = cmul(Ev[j], x[j]);
            Sp[o] = caxpy(Sv[j], T(2), Ek3);
            x[j] = cadd(D, caxpy(cmul(ev[j], D), h, Ek3));
        } else {
            const cx<T> e2 = ev[j];
            cx<T> L = Dl[j];
            cx<T> d = cmul(e2, D);
            if constexpr (COMP)
                d = cadd(d, cmul(e2, L));
            d = caxpy(d, h6, cadd(Sv[j], x[j]));
            accumulate<T, COMP>(D, L, d);
            if (valid) {
                hi[o] = D;
                if constexpr (COMP)
                    lo[o] = L;
                if (!(isfinite(D.re) && isfinite(D.im)))
                    A.status[inst] = 1;
            }
            x[j] = D;
        }
    }
    if (st == LARGE_FINAL)
        return;
    // inverse transform over m1 of the next stage input, twiddle, store Y column m2
    grp.inverse(x, 0);
    if (valid) {
        cx<T>* y = reinterpret_cast<cx<T>*>(A.Y) + ibase + (long long)m2 * N1 + t;
#pragma unroll
        for (int j = 0; j < R; ++j)
            y[j * P] = cmul(x[j], w[j]);   // * exp(+2 pi i j1 m2 / N)
    }
}

// ----------------------------------------------------------------------------------------
// One launch for a whole call: the row and column passes of every stage of every step run in
// one kernel whose blocks meet at grid-wide barriers instead of kernel boundaries.  Block b
// owns column m2 = b mod N2 of instance b / N2 for the whole launch, so that column's field
// (hi and compensation word) and Runge-Kutta accumulator stay in registers across steps, and
// its output twiddles with them; in the row passes the same block takes rows b G .. b G + G - 1
// (G = N1 / N2 rows of N2 / R threads: every block has N1 / R threads in both passes).  Only the
// inter-pass buffers Y and Z go through memory, read past L1 (ld.global.cg: other SMs wrote
// them since the last barrier).  Every block must be resident at once: the host launches it
// cooperatively, on request (persistent = 2) and only where the occupancy allows it.  The
// arithmetic is that of the row and column kernels above, expression for expression, so both
// paths give the same bits.  On N = 2^17 it takes 30.7 us per step against 29.6 for the kernel
// sequence: a block spends its time at the barriers waiting for the slowest block and, in the
// fence before its arrival, for its stores (ncu: barrier, long-scoreboard and membar stalls
// first), as the kernels of the sequence wait for them at exit.
//
// Barrier: the block's threads synchronise; thread 0 issues a GPU-scope fence (cumulative over
// the block's writes ordered before it by the block barrier), adds one arrival to a 64-bit
// counter, polls it until it reaches k x (blocks) for the k-th barrier of the launch, and
// fences again before the block barrier that releases the other threads.  The poll is bounded: a block that gives up
// reports status 2 for its column's instance and returns, and the others then give up at
// their next barrier, so every wait ends.
// ----------------------------------------------------------------------------------------
CME_DEV unsigned long long ld_relaxed_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

CME_DEV bool grid_barrier(unsigned long long* ctr, unsigned long long target, int tries, int* ok)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        // release: the fence orders the block's earlier writes (through the block barrier)
        // before the arrival, which is a reduction without a returned value
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        asm volatile("red.relaxed.gpu.global.add.u64 [%0], 1;" ::"l"(ctr) : "memory");
        bool done = false;
        for (int k = 0; k < tries && !done; ++k)
            done = ld_relaxed_u64(ctr) >= target;
        // acquire: later reads of the block (through the block barrier) after the observation
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        *ok = done;
    }
    __syncthreads();
    return *ok != 0;
}

template <typename T>
CME_DEV cx<T> ldcg(const cx<T>* p)
{
    const typename v2<T>::type v = __ldcg(reinterpret_cast<const typename v2<T>::type*>(p));
    return {v.x, v.y};
}

template <typename T, int LOGN1, int LOGN2, int R>
constexpr size_t large_grid_smem()
{
    return group_smem_bytes(sizeof(T), LOGN1, R) +
           (size_t)(Plan<LOGN1, R>::P / Plan<LOGN2, R>::P) * group_smem_bytes(sizeof(T), LOGN2, R);
}

template <typename T, int LOGN1, int LOGN2, int R>
__global__ void __launch_bounds__(Plan<LOGN1, R>::P) large_grid_kernel(const LargeArgs A)
{
    using GC = Group<T, LOGN1, R>;
    using GW = Group<T, LOGN2, R>;
    constexpr int N1 = GC::N, PC = GC::P, N2 = GW::N, PR = GW::P, GR = PC / PR;
    static_assert(GR * PR == PC && (GR == 1 || GR == 2), "N1 = N2 or 2 N2");
    constexpr long long N = (long long)N1 * N2;
    constexpr bool COMP = GC::COMP;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int bar_ok;
    const int tid = threadIdx.x;
    // column pass: column m2 of instance ci
    const int ci = (int)(blockIdx.x / N2);
    const int m2 = (int)(blockIdx.x - (unsigned)ci * N2);
    // row pass: row blockIdx.x G + g of the instance-major row list
    const int g = tid / PR;
    const long long row = (long long)blockIdx.x * GR + g;
    const int ri = (int)(row / N1);
    const int j1 = (int)(row - (long long)ri * N1);
    GC gc;
    gc.setup(smem, 0, tid, A.tw1);
    GW gw;
    gw.setup(smem + group_smem_bytes(sizeof(T), LOGN1, R), g, tid - g * PR, A.tw2);
    const int t = gc.t, tr = gw.t;

    const long long ibase = (long long)ci * N;
    const long long e0 = ibase + (long long)m2 * N1 + t;   // column element j at e0 + j PC
    const long long f0 = A.base + e0;
    cx<T>* hi = reinterpret_cast<cx<T>*>(A.hi) + f0;
    cx<T>* lo = reinterpret_cast<cx<T>*>(A.lo) + f0;
    const cx<T>* Ep = reinterpret_cast<const cx<T>*>(A.E) + f0;
    const cx<T>* e1p = reinterpret_cast<const cx<T>*>(A.e1) + f0;
    const cx<T>* e2p = reinterpret_cast<const cx<T>*>(A.e2) + f0;
    cx<T> Dh[R], Dl[R], Sv[R], wc[R], wr[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        Dh[j] = hi[j * PC];
        Dl[j] = COMP ? lo[j * PC] : cx<T>{T(0), T(0)};
        Sv[j] = cx<T>{T(0), T(0)};
        wc[j] = gload<T>(A.twN, ((long long)(t + j * PC) * m2) & (N - 1));
        wr[j] = gload<T>(A.twN, ((long long)j1 * (tr + j * PR)) & (N - 1));
    }
    const T gNr = (T)A.g0[ri] * ((T)1 / (T)N);
    T h, hh, h6;
    if constexpr (sizeof(T) == 4) {
        h = A.hf;
        hh = A.hhf;
        h6 = A.h6f;
    } else {
        h = A.h;
        hh = 0.5 * A.h;
        h6 = A.h / 6.0;
    }
    // Y column-major, Z row-major, as for the kernel sequence: contiguous stores
    cx<T>* ycol = reinterpret_cast<cx<T>*>(A.Y) + ibase + (long long)m2 * N1 + t;
    const cx<T>* yrow = reinterpret_cast<const cx<T>*>(A.Y) + (long long)ri * N +
                        (long long)tr * N1 + j1;
    cx<T>* zrow = reinterpret_cast<cx<T>*>(A.Z) + (long long)ri * N + (long long)j1 * N2 + tr;
    const cx<T>* zcol = reinterpret_cast<const cx<T>*>(A.Z) + ibase + (long long)t * N2 + m2;

    const unsigned long long nb = gridDim.x;
    const int tries = A.bar_fault ? 1024 : (1 << 22);
    unsigned long long nbar = 0;
    auto barrier = [&]() {
        ++nbar;
        return grid_barrier(A.bar, nbar * nb + (A.bar_fault ? 1 : 0), tries, &bar_ok);
    };
    // the inverse transform over m1 of a stage input, twiddle, store Y column m2
    auto col_out = [&](cx<T>(&x)[R]) {
        gc.inverse(x, 0);
#pragma unroll
        for (int j = 0; j < R; ++j)
            ycol[j * PC] = cmul(x[j], wc[j]);   // * exp(+2 pi i j1 m2 / N)
    };

    bool ok;
    {
        cx<T> x[R];
#pragma unroll
        for (int j = 0; j < R; ++j)
            x[j] = Dh[j];
        col_out(x);
        ok = barrier();
    }
    for (long long s = 0; s < A.nsteps && ok; ++s) {
#pragma unroll 1
        for (int st = 0; st < 4; ++st) {
            // row pass: inverse over m2, Kerr term, forward over j2, twiddle, store Z
            {
                cx<T> x[R];
#pragma unroll
                for (int j = 0; j < R; ++j)
                    x[j] = ldcg(yrow + (long long)j * PR * N1);
                gw.rhs(x, gNr, cx<T>{T(0), T(0)});
#pragma unroll
                for (int j = 0; j < R; ++j)
                    zrow[j * PR] = cmulc(x[j], wr[j]);   // * exp(-2 pi i j1 m2/N)
            }
            if (!(ok = barrier()))
                break;
            // column pass: forward over j1, Kerr factors, padding mask, pump
            cx<T> x[R];
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const cx<T> v = ldcg(zcol + (long long)j * PC * N2);
                x[j] = {v.re, -v.im};
            }
            gc.inverse(x, 1);
#pragma unroll
            for (int j = 0; j < R; ++j)
                x[j].im = -x[j].im;
            if (A.kerr) {
                const T* km = reinterpret_cast<const T*>(A.kerr) + f0;
#pragma unroll
                for (int j = 0; j < R; ++j)
                    x[j] = cscale(x[j], __ldg(km + j * PC));
            }
            if (A.phys) {
                const int M = A.phys[ci];
                if (M < N) {
                    const long long mlo = -(M / 2), mhi = M - M / 2 - 1;
#pragma unroll
                    for (int j = 0; j < R; ++j) {
                        const long long m = (long long)(t + j * PC) * N2 + m2;
                        const long long mu = m >= N / 2 ? m - N : m;
                        if (mu < mlo || mu > mhi)
                            x[j] = cx<T>{T(0), T(0)};
                    }
                }
            }
            if (t == 0 && m2 == 0) {
                const double2 pd = A.pump[ci];
                x[0] = cadd(x[0], cx<T>{(T)pd.x, (T)pd.y});
            }
            // Runge-Kutta combination of stage st and the next stage's input
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const cx<T> D = Dh[j];
                if (st == 0) {
                    const cx<T> Ev = gload<T>(Ep, j * PC), ev = gload<T>(e1p, j * PC);
                    const cx<T> k1 = cmul(Ev, x[j]);
                    Sv[j] = cmul(Ev, k1);
                    x[j] = cadd(D, caxpy(cmul(ev, D), hh, k1));
                } else if (st == 1) {
                    const cx<T> Ev = gload<T>(Ep, j * PC), ev = gload<T>(e1p, j * PC);
                    Sv[j] = caxpy(Sv[j], T(2), cmul(Ev, x[j]));
                    x[j] = cadd(D, caxpy(cmul(ev, D), hh, x[j]));
                } else if (st == 2) {
                    const cx<T> Ev = gload<T>(Ep, j * PC), ev = gload<T>(e2p, j * PC);
                    const cx<T> Ek3 = cmul(Ev, x[j]);
                    Sv[j] = caxpy(Sv[j], T(2), Ek3);
                    x[j] = cadd(D, caxpy(cmul(ev, D), h, Ek3));
                } else {
                    const cx<T> e2 = gload<T>(e2p, j * PC);
                    cx<T> L = Dl[j];
                    cx<T> Dn = D;
                    cx<T> d = cmul(e2, D);
                    if constexpr (COMP)
                        d = cadd(d, cmul(e2, L));
                    d = caxpy(d, h6, cadd(Sv[j], x[j]));
                    accumulate<T, COMP>(Dn, L, d);
                    Dh[j] = Dn;
                    Dl[j] = L;
                    if (!(isfinite(Dn.re) && isfinite(Dn.im)))
                        A.status[ci] = 1;
                    x[j] = Dn;
                }
            }
            if (st == 3 && s == A.nsteps - 1)
                break;   // the last step's field stays in registers until the store below
            col_out(x);
            if (!(ok = barrier()))
                break;
        }
    }
#pragma unroll
    for (int j = 0; j < R; ++j) {
        hi[j * PC] = Dh[j];
        if constexpr (COMP)
            lo[j * PC] = Dl[j];
    }
    if (!ok && tid == 0)
        A.status[ci] = 2;
}

}  // namespace cme
