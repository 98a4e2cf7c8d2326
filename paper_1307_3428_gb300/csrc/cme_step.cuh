// Persistent step kernels: one launch advances every instance of a uniform-N group by nsteps
// RK4IP or Strang steps with the field held in registers throughout.
#pragma once

#include <type_traits>

#include "cme_core.cuh"

namespace cme {

// Threads per block a kernel is compiled for: groups of P >= 64 threads run one instance per
// block (so the register file is shared by as few threads as possible); narrower groups pack
// up to 256 threads.
template <int LOGN, int R>
constexpr int max_threads() { return Plan<LOGN, R>::P >= 64 ? Plan<LOGN, R>::P : 256; }

// Per-mode propagators of the RK4IP and Strang steps: E = exp(L h/2), e1 = expm1(L h/2),
// e2 = expm1(L h).  For FP32 groups up to N = 1024 they are held in registers for the whole
// launch; otherwise they are read through the read-only cache where used.
template <typename T, int LOGN, int R, int C = 1>
struct Props {
    // cluster groups run few threads per block, so their register budget has room, and so do
    // 16-value groups of N >= 2048, whose twiddles live in shared memory
    static constexpr bool IN_REGS =
        sizeof(T) == 4 && (((LOGN <= 10 || C > 1) && R <= 8) || (LOGN >= 11 && R == 16));
    cx<T> E[IN_REGS ? R : 1], e1[IN_REGS ? R : 1], e2[IN_REGS ? R : 1];
    const cx<T>* pE;   // pointers pre-offset to (instance offset + t)
    const cx<T>* pe1;
    const cx<T>* pe2;

    CME_DEV void init(const StepArgs& a, long long off, int t)
    {
        constexpr int P = Plan<LOGN, R>::P;
        pE = reinterpret_cast<const cx<T>*>(a.E) + off + t;
        pe1 = reinterpret_cast<const cx<T>*>(a.e1) + off + t;
        pe2 = reinterpret_cast<const cx<T>*>(a.e2) + off + t;
        if constexpr (IN_REGS) {
#pragma unroll
            for (int j = 0; j < R; ++j) {
                E[j] = gload<T>(pE, j * P);
                e1[j] = gload<T>(pe1, j * P);
                e2[j] = gload<T>(pe2, j * P);
            }
        }
    }
    CME_DEV cx<T> getE(int j) const
    {
        if constexpr (IN_REGS)
            return E[j];
        else
            return gload<T>(pE, j * Plan<LOGN, R>::P);
    }
    CME_DEV cx<T> get1(int j) const
    {
        if constexpr (IN_REGS)
            return e1[j];
        else
            return gload<T>(pe1, j * Plan<LOGN, R>::P);
    }
    CME_DEV cx<T> get2(int j) const
    {
        if constexpr (IN_REGS)
            return e2[j];
        else
            return gload<T>(pe2, j * Plan<LOGN, R>::P);
    }
};

// Twiddles stay in registers up to N = 1024 (FP32) / 512 (FP64).
template <typename T, int LOGN>
constexpr bool twiddles_in_regs() { return sizeof(T) == 4 ? LOGN <= 10 : LOGN <= 9; }

// The transform of a group: one block's Stockham transform, or for C > 1 the four-step
// cluster transform and its transform inside one block.
template <typename T, int LOGN, int R, int C>
struct GroupFFT {
    using CF = ClusterFFT<T, LOGN, R, C>;
    using TF = typename CF::TL;
};
template <typename T, int LOGN, int R>
struct GroupFFT<T, LOGN, R, 1> {
    using CF = void;
    using TF = Transform<T, LOGN, R, (Plan<LOGN, R>::P <= 32)>;
};

// Per-thread view of one instance: the transform machinery plus the instance constants.
// C > 1: the instance is spread over the C blocks of a thread-block cluster.
template <typename T, int LOGN, int R, int C = 1>
struct Group {
    using PL = Plan<LOGN, R>;
    static constexpr int N = PL::N, P = PL::P;
    static constexpr bool WARP = (C == 1 && P <= 32);
    static constexpr bool COMP = (sizeof(T) == 4);  // compensated state in FP32
    // C > 1: the four-step cluster transform; TF is then its transform inside one block
    using CF = typename GroupFFT<T, LOGN, R, C>::CF;
    using TF = typename GroupFFT<T, LOGN, R, C>::TF;
    static constexpr int LC = ilog2(C);
    // twiddles: registers (small N), this group's shared memory (FP32 one-block groups of
    // N >= 2048), else the global table (read at stride C by the block transforms of a cluster)
    static constexpr bool TW_REGS =
        twiddles_in_regs<T, LOGN - LC>() && (C == 1 || sizeof(T) == 4);
    static constexpr bool TW_SMEM = !TW_REGS && twiddles_in_smem(sizeof(T), LOGN - LC);
    using TW = std::conditional_t<TW_SMEM, TwiddlesSmem<T, LOGN - LC, R, C>,
                                  Twiddles<T, LOGN - LC, R, TW_REGS, C>>;

    int t;         // the thread holds modes t + jP
    int ts;        // this thread's slots ts + jP of per-thread scratch vectors (coalesced)
    int par;
    Xbuf<T> buf;   // first of the two ping-pong exchange buffers
    typename TF::Addr ad;
    TW tw;

    // C > 1: all-to-all state (block `rank`, thread l): this thread's slots of the receive
    // buffer 0; shared::cluster address of receive buffer 0 and of its mbarrier in every
    // block; byte offsets of this thread's stores; the twiddles of the two directions in this
    // block's shared memory (thread-major); the receive-buffer parity; the phase parities of
    // this block's two mbarriers; whether a wait gave up.
    Xbuf<T> abuf;
    uint32_t rb[C > 1 ? C : 1];
    uint32_t rmb[C > 1 ? C : 1];
    uint32_t mb;
    uint32_t om, ot;
    const cx<T>* twm;
    const cx<T>* twt;
    int apar;
    uint32_t ph;
    bool timed_out;
    int fault;     // StepArgs::a2a_fault
    // polls of one all-to-all wait before it gives up (a wait normally ends within a few)
    static constexpr int WAIT_TRIES = 1 << 20;

    // a bounded wait of an all-to-all gave up (the results are then not valid)
    CME_DEV bool failed() const
    {
        if constexpr (C == 1)
            return false;
        else
            return timed_out;
    }
    // Physical modes (the zero padding of Sec. 2): of the N modes only the centred M,
    // mu = mlo .. mhi, are physical; the right-hand side is zero on the others, which stay at
    // zero.  masked = false (M = N) skips the test.
    bool masked;
    int mlo, mhi;

    CME_DEV void set_modes(int M)
    {
        masked = M < N;
        mlo = -(M / 2);
        mhi = M - M / 2 - 1;
    }
    // Is the thread's position t + jP (mode mu = p or p - N, transform order) physical?
    CME_DEV bool physical(int j) const
    {
        if (!masked)
            return true;
        const int p = t + j * P;
        const int mu = p >= N / 2 ? p - N : p;
        return mu >= mlo && mu <= mhi;
    }
    CME_DEV void mask(cx<T> (&x)[R]) const
    {
        if (masked) {
#pragma unroll
            for (int j = 0; j < R; ++j)
                if (!physical(j))
                    x[j] = cx<T>{T(0), T(0)};
        }
    }
    // Per-mode Kerr coefficient (Sec. 2: g0 need not be constant): the four-wave-mixing term
    // of output mode mu carries g0_mu instead of the instance's g0, applied as the factor
    // km[j P] of this thread's mode t + jP to the forward transform's output (the instance's g0
    // is then 1).  km = null (the default) leaves every mode at g0.
    const T* km;
    CME_DEV void set_kerr(const void* table, long long off)
    {
        km = table ? reinterpret_cast<const T*>(table) + off + t : nullptr;
    }
    // The right-hand side's output side: the per-mode Kerr factor, then the physical-mode mask.
    CME_DEV void out_modes(cx<T> (&x)[R]) const
    {
        if (km) {
#pragma unroll
            for (int j = 0; j < R; ++j)
                x[j] = cscale(x[j], __ldg(km + j * P));
        }
        mask(x);
    }

    // The step loops contain a single copy of the transform code (instruction-cache
    // footprint): the forward transform is computed as conj(inverse(conj(x))).  d = 0 takes
    // modes to time samples, d = 1 time samples to modes (the same for one block; the
    // reverse order of the stages for a cluster).
    CME_DEV void inverse(cx<T> (&x)[R], int d)
    {
        if constexpr (C == 1) {
            TF::template run<+1>(x, tw, buf, par, ad);
        } else {
            if (d == 1) {
                CF::radix_c(x);
                twiddle(x, twt);
                all_to_all<true>(x);
            }
            TF::template run<+1>(x, tw, buf, par, ad);
            if (d == 0) {
                twiddle(x, twm);
                all_to_all<false>(x);
                CF::radix_c(x);
            }
        }
    }
    CME_DEV static void twiddle(cx<T> (&x)[R], const cx<T>* w)
    {
#pragma unroll
        for (int j = 0; j < R; ++j)
            x[j] = cmul(x[j], w[j * CF::PC]);
    }
    // Cluster all-to-all.  Modes to time (T2M = false): the value of local position
    // n2 = l + PC j (k1 = rank) goes to block j mod C, slot rank G + j / C.  Time to modes:
    // slot i = k1 G + m of thread (rank, l) goes to block k1, slot rank + C m.  Every thread
    // reads its slots j at l + PC j of its own buffer.
    template <bool T2M>
    CME_DEV void all_to_all(cx<T> (&x)[R])
    {
        constexpr int PC = CF::PC, G = CF::G, W = Xbuf<T>::words_per_elem;
        if (timed_out) {
            // after a wait gave up this thread stores, arrives and waits no more, so no
            // mbarrier receives an arrival or bytes beyond the phase it is stuck in
            apar ^= 1;
            return;
        }
        const uint32_t po = (uint32_t)apar * (uint32_t)(CF::N2 * 8 * W);
        const uint32_t bo = 8u * (uint32_t)apar;   // mbarrier of buffer apar
#pragma unroll
        for (int j = 0; j < R; ++j) {
            if constexpr (T2M)
                abuf.put_remote_async(rb[j / G] + ot + po + (uint32_t)(8 * PC * C * (j % G)),
                                      x[j], rmb[j / G] + bo);
            else
                abuf.put_remote_async(rb[j % C] + om + po + (uint32_t)(8 * PC * (j / C)), x[j],
                                      rmb[j % C] + bo);
        }
        // the phase ends when this block's one arrival is in and all N2 values have landed
        if (threadIdx.x == 0)
            mbar_arrive_expect_tx(mb + bo, (uint32_t)(CF::N2 * 8 * W + (fault ? 8 : 0)));
        if (!mbar_wait(mb + bo, (ph >> apar) & 1u, fault ? 1024 : WAIT_TRIES))
            timed_out = true;   // the caller reports the instance
        ph ^= 1u << apar;
        const Xbuf<T> mine = abuf.at(apar * CF::N2);
#pragma unroll
        for (int j = 0; j < R; ++j)
            x[j] = mine.get(PC * j);
        apar ^= 1;
    }

    // F(x) = pump + i (g0/N) DFT(|a|^2 a), a = inverse transform of x   (Eq. 4)
    CME_DEV void rhs(cx<T> (&x)[R], T gN, cx<T> pump) { rhs_store_a(x, gN, pump, nullptr); }

    // The same, also storing the time-domain field a at aout[j P] unless aout is null.
    CME_DEV void rhs_store_a(cx<T> (&x)[R], T gN, cx<T> pump, cx<T>* aout)
    {
#pragma unroll 1
        for (int d = 0; d < 2; ++d) {
            inverse(x, d);
            if (d == 0 && aout) {
#pragma unroll
                for (int j = 0; j < R; ++j)
                    sstore(aout + j * P, x[j]);
            }
            if (d == 0) {
                // conj(i c a) with c = (g0/N) |a|^2
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    const T c = gN * (x[j].re * x[j].re + x[j].im * x[j].im);
                    x[j] = {-c * x[j].im, -c * x[j].re};
                }
            }
        }
#pragma unroll
        for (int j = 0; j < R; ++j)
            x[j].im = -x[j].im;
        out_modes(x);
        if (t == 0)
            x[0] = cadd(x[0], pump);
    }

    static constexpr bool ACC_SMEM = C == 1 && acc_in_smem(sizeof(T), LOGN, R);
    cx<T>* accS;   // shared-memory accumulator S (ACC_SMEM), pre-offset by t
    cx<T>* accL;   // shared-memory compensation word (ACC_SMEM, FP32), pre-offset by t

    // Block-local set-up: thread index in the group, exchange buffers, addresses, twiddles.
    CME_DEV void setup(unsigned char* smem, int g, int t_, const void* tw_table)
    {
        constexpr int W = Xbuf<T>::words_per_elem;  // 8-byte words per element
        unsigned char* gbase = smem + (size_t)g * group_smem_bytes(sizeof(T), LOGN, R);
        double* base = reinterpret_cast<double*>(gbase);
        cx<T>* acc = reinterpret_cast<cx<T>*>(gbase + (size_t)2 * W * PL::BUF * 8);
        static_assert(xbuf_bytes(sizeof(T), LOGN) == (size_t)2 * W * PL::BUF * 8, "layout");
        accS = acc + t_;
        accL = acc + N + t_;
        if constexpr (sizeof(T) == 4) {
            buf.p = reinterpret_cast<float2*>(base);
        } else {
            buf.re = base;           // buffer 0: re [0, BUF), im [BUF, 2 BUF)
            buf.stride = PL::BUF;    // buffer 1 starts at 2 BUF (Xbuf::at)
        }
        t = t_;
        ts = t_;
        par = 0;
        ad = TF::make_addr(t);
        if constexpr (TW_SMEM)
            tw.init(tw_table, t,
                    reinterpret_cast<cx<T>*>(gbase + xbuf_bytes(sizeof(T), LOGN) +
                                             acc_bytes(sizeof(T), LOGN, R)));
        else
            tw.init(tw_table, t);
        set_modes(N);
        km = nullptr;
    }

    // Cluster set-up (C > 1): block `rank` of the cluster, thread l of the block.  The block's
    // dynamic shared memory holds the two exchange buffers of its N2-point transform, the two
    // all-to-all receive buffers, the two twiddle arrays of the four-step transform, (FP32,
    // N2 >= 2048) the pass twiddles of the N2-point transform, and the receive buffers' two
    // mbarriers (its last 16 bytes).
    CME_DEV void setup_cluster(unsigned char* smem, int rank, int l, const void* tw_table,
                               int a2a_fault)
    {
        static_assert(C > 1, "cluster groups only");
        constexpr int W = Xbuf<T>::words_per_elem, PC = CF::PC, N2 = CF::N2, G = CF::G;
        unsigned char* a2a = smem + (size_t)2 * TF::BUF * 8 * W;
        cx<T>* tws = reinterpret_cast<cx<T>*>(a2a + (size_t)2 * N2 * 8 * W);
        if constexpr (sizeof(T) == 4) {
            buf.p = reinterpret_cast<float2*>(smem);
            abuf.p = reinterpret_cast<float2*>(a2a) + l;
        } else {
            buf.re = reinterpret_cast<double*>(smem);
            buf.stride = TF::BUF;
            abuf.re = reinterpret_cast<double*>(a2a) + l;
            abuf.stride = N2;
        }
        accS = nullptr;
        accL = nullptr;
        t = rank + C * l;
        ts = rank * PC + l;
        par = 0;
        apar = 0;
        ad = TF::make_addr(l);
        if constexpr (TW_SMEM)
            tw.init(tw_table, l, tws + 2 * N2);
        else
            tw.init(tw_table, l);
        const uint32_t a0 = smem_addr(a2a);
        mb = smem_addr(reinterpret_cast<unsigned char*>(tws + 2 * N2) +
                       (TW_SMEM ? tw_bytes(sizeof(T), LOGN - LC, R) : 0));
#pragma unroll
        for (int c = 0; c < C; ++c) {
            rb[c] = dsmem_map(a0, c);
            rmb[c] = dsmem_map(mb, c);
        }
        // the kernel's cluster barrier before the first all-to-all publishes the initialisation
        if (l == 0) {
            mbar_init(mb, 1);
            mbar_init(mb + 8u, 1);
            mbar_init_fence();
        }
        ph = 0;
        timed_out = false;
        fault = a2a_fault;
        om = 8u * (uint32_t)(l + PC * rank * G);
        ot = 8u * (uint32_t)(l + PC * rank);
        // exp(2 pi i n2 k1 / N): after the block transform (n2 = l + PC j, k1 = rank), and
        // after the C-point transforms (n2 = rank PC + l + P (i mod G), k1 = i / G)
        const int tp = rank * PC + l;
        cx<T>* wm = tws + l;
        cx<T>* wt = tws + N2 + l;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            wm[j * PC] = gload<T>(tw_table, ((l + PC * j) * rank) & (N - 1));
            wt[j * PC] = gload<T>(tw_table, ((tp + P * (j % G)) * (j / G)) & (N - 1));
        }
        twm = wm;
        twt = wt;
        set_modes(N);
        km = nullptr;
    }
};

// Dynamic shared memory of one block of a cluster group: two exchange buffers.
template <typename T, int LOGN, int R, int C>
CME_HD constexpr size_t cluster_smem_bytes()
{
    using CF = ClusterFFT<T, LOGN, R, C>;
    constexpr size_t W = Xbuf<T>::words_per_elem;
    return (size_t)2 * CF::TL::BUF * 8 * W + (size_t)2 * CF::N2 * 8 * W +
           (size_t)2 * CF::N2 * sizeof(cx<T>) +
           (Group<T, LOGN, R, C>::TW_SMEM ? tw_bytes(sizeof(T), LOGN - CF::LC, R) : 0) + 16;
}

template <typename T>
struct Coef;  // step coefficients in the field precision, converted once on the host
template <>
struct Coef<float> {
    CME_DEV static float h(const StepArgs& a) { return a.hf; }
    CME_DEV static float hh(const StepArgs& a) { return a.hhf; }
    CME_DEV static float h6(const StepArgs& a) { return a.h6f; }
};
template <>
struct Coef<double> {
    CME_DEV static double h(const StepArgs& a) { return a.h; }
    CME_DEV static double hh(const StepArgs& a) { return 0.5 * a.h; }
    CME_DEV static double h6(const StepArgs& a) { return a.h / 6.0; }
};

// nsteps steps of the instances [first, first + blockDim.x / P) of the group described by a
// (group-relative indices; groups past a.ninst recompute the last instance and store nothing).
// The evolving field of one thread: hi part in registers; the compensation word Dl (FP32) and
// the Runge-Kutta accumulator S in registers, or (ACC_SMEM) in this thread's own shared-memory
// slots t + jP.
template <typename T, int LOGN, int R, int C = 1>
struct FieldState {
    using GR = Group<T, LOGN, R, C>;
    static constexpr int P = GR::P;
    static constexpr bool COMP = GR::COMP, AS = GR::ACC_SMEM;
    cx<T> Dh[R];
    cx<T> Dlr[AS ? 1 : R];
    cx<T> Sr[AS ? 1 : R];
    cx<T>* accL;
    cx<T>* accS;

    CME_DEV void bind(const GR& grp)
    {
        accL = grp.accL;
        accS = grp.accS;
    }
    CME_DEV cx<T> getL(int j) const
    {
        if constexpr (!COMP)
            return cx<T>{T(0), T(0)};
        else if constexpr (AS)
            return accL[j * P];
        else
            return Dlr[j];
    }
    CME_DEV void setL(int j, cx<T> v)
    {
        if constexpr (COMP) {
            if constexpr (AS)
                accL[j * P] = v;
            else
                Dlr[j] = v;
        }
    }
    CME_DEV cx<T> getS(int j) const
    {
        if constexpr (AS)
            return accS[j * P];
        else
            return Sr[j];
    }
    CME_DEV void setS(int j, cx<T> v)
    {
        if constexpr (AS)
            accS[j * P] = v;
        else
            Sr[j] = v;
    }
    // D += d (compensated two-sum in FP32)
    CME_DEV void add(int j, cx<T> d)
    {
        cx<T> l = getL(j);
        accumulate<T, COMP>(Dh[j], l, d);
        setL(j, l);
    }
    CME_DEV void load(const cx<T>* hi, const cx<T>* lo)
    {
#pragma unroll
        for (int j = 0; j < R; ++j) {
            Dh[j] = hi[j * P];
            if constexpr (COMP)
                setL(j, lo[j * P]);
        }
    }
    CME_DEV void store(cx<T>* hi, cx<T>* lo) const
    {
#pragma unroll
        for (int j = 0; j < R; ++j) {
            hi[j * P] = Dh[j];
            if constexpr (COMP)
                lo[j * P] = getL(j);
        }
    }
};

// Instance constants of the step loops.
template <typename T>
struct StepConsts {
    cx<T> pump;   // sqrt(kappa_ext) A_in
    cx<T> cp;     // Strang pump increment over h/2
    cx<T> cp2;    // ... over h
    T gN;         // g0 / N
    T g0h;        // g0 h / 2 (Strang half phase per |a|^2)
    T h, hh, h6;
};

// One RK4IP step (Sec. 2 "fourth-order Runge-Kutta"; Hult 2007) written as increments of D:
//   x2 = D + (e1 D + h/2 k1),  x3 = D + (e1 D + h/2 k2),  x4 = D + (e2 D + h E k3),
//   D' = D + e2 D + h/6 [E (k1 + 2 k2 + 2 k3) + k4],  k1 = E F(D),  k_i = F(x_i),
// with E = exp(L h/2), e1 = expm1(L h/2), e2 = expm1(L h).  The four stages share one copy of
// the right-hand-side code (a runtime loop).
// STAGES = true also stores, unless so is null (the adjoint's recomputation), the right-hand-side
// values y1 = F(D), k2 = F(x2), k3 = F(x3) of the thread's positions at so[st * sstride + j P],
// st = 0, 1, 2, and the time-domain fields a of the four stage inputs D, x2, x3, x4 at
// so[(3 + st) * sstride + j P], st = 0..3.
template <bool STAGES, bool CACHE = false, typename T, int LOGN, int R, int C>
CME_DEV void rk4ip_step_impl(Group<T, LOGN, R, C>& grp, FieldState<T, LOGN, R, C>& fs,
                             const Props<T, LOGN, R, C>& pr, const StepConsts<T>& c, cx<T>* so,
                             long long sstride)
{
    constexpr bool COMP = Group<T, LOGN, R, C>::COMP;
    constexpr int P = Group<T, LOGN, R, C>::P;
    cx<T> x[R];
    // CACHE: e1 D (stages 0, 1), then e2 D (stages 2, 3) computed once and kept in registers
    // across the stage's transforms (kernels with registers to spare); else recomputed
    cx<T> eD[CACHE ? R : 1];
#pragma unroll
    for (int j = 0; j < R; ++j)
        x[j] = fs.Dh[j];
    // one RK stage (st = 0 ... 3)
    auto stage = [&](int st) {
        if constexpr (STAGES)
            grp.rhs_store_a(x, c.gN, c.pump, so ? so + (3 + st) * sstride : nullptr);
        else
            grp.rhs(x, c.gN, c.pump);
        if constexpr (STAGES) {
            if (st < 3 && so) {
#pragma unroll
                for (int j = 0; j < R; ++j)
                    sstore(so + st * sstride + j * P, x[j]);
            }
        }
        if (st == 0) {
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const cx<T> E = pr.getE(j);
                const cx<T> k1 = cmul(E, x[j]);
                fs.setS(j, cmul(E, k1));
                const cx<T> e1D = cmul(pr.get1(j), fs.Dh[j]);
                if constexpr (CACHE)
                    eD[j] = e1D;
                x[j] = cadd(fs.Dh[j], caxpy(e1D, c.hh, k1));
            }
        } else if (st == 1) {
#pragma unroll
            for (int j = 0; j < R; ++j) {
                fs.setS(j, caxpy(fs.getS(j), T(2), cmul(pr.getE(j), x[j])));
                cx<T> e1D;
                if constexpr (CACHE)
                    e1D = eD[j];
                else
                    e1D = cmul(pr.get1(j), fs.Dh[j]);
                x[j] = cadd(fs.Dh[j], caxpy(e1D, c.hh, x[j]));
            }
        } else if (st == 2) {
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const cx<T> Ek3 = cmul(pr.getE(j), x[j]);
                fs.setS(j, caxpy(fs.getS(j), T(2), Ek3));
                const cx<T> e2D = cmul(pr.get2(j), fs.Dh[j]);
                if constexpr (CACHE)
                    eD[j] = e2D;
                x[j] = cadd(fs.Dh[j], caxpy(e2D, c.h, Ek3));
            }
        } else {
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const cx<T> e2 = pr.get2(j);
                cx<T> d;
                if constexpr (CACHE)
                    d = eD[j];
                else
                    d = cmul(e2, fs.Dh[j]);
                if constexpr (COMP)
                    d = cadd(d, cmul(e2, fs.getL(j)));
                d = caxpy(d, c.h6, cadd(fs.getS(j), x[j]));
                fs.add(j, d);
            }
        }
    };
    // One-block CACHE kernels (registers to spare) take the four stages unrolled: 51.6 -> 49.4
    // ms per headline run.  Elsewhere one copy of the stage code in a loop keeps the
    // instruction footprint small: unrolled, the 8-block cluster kernel of N = 4096 took 6.9
    // instead of 5.1 us per step.
    if constexpr (CACHE && C == 1) {
#pragma unroll
        for (int st = 0; st < 4; ++st)
            stage(st);
    } else {
#pragma unroll 1
        for (int st = 0; st < 4; ++st)
            stage(st);
    }
}

// Whether a step kernel has the registers to keep e1 D / e2 D across a stage (FP32 at 8 values
// per thread, at most 256 threads per block: N = 512, 64 threads, 168 -> 192 registers), not
// in the work-list kernel, whose tiles share one register budget.
template <typename T, int LOGN, int R, int C>
CME_HD constexpr bool rk_cache_ed()
{
    return sizeof(T) == 4 && R <= 8 && Plan<LOGN, R>::P / C <= 256;
}

template <bool CACHE = false, typename T, int LOGN, int R, int C>
CME_DEV void rk4ip_step(Group<T, LOGN, R, C>& grp, FieldState<T, LOGN, R, C>& fs,
                        const Props<T, LOGN, R, C>& pr, const StepConsts<T>& c)
{
    rk4ip_step_impl<false, CACHE>(grp, fs, pr, c, static_cast<cx<T>*>(nullptr), 0);
}

// sin y and cos y in FP32 for the Strang Kerr phase y = g0 |a|^2 h / 2, which is small in any
// resolved step.  For |y| <= 1/2 the Taylor series of sin (to y^9) and cos (to y^8), evaluated
// in y^2 by Horner's rule, leave truncation errors below y^11/11! <= 1.2e-11 and
// y^10/10! <= 2.7e-10, far under FP32 rounding; larger |y| (small_phase false) take sincosf.
CME_DEV void taylor_sincos(float y, float& s, float& c)
{
    const float y2 = y * y;
    s = y * (1.f + y2 * (-1.f / 6 + y2 * (1.f / 120 + y2 * (-1.f / 5040 + y2 * (1.f / 362880)))));
    c = 1.f + y2 * (-0.5f + y2 * (1.f / 24 + y2 * (-1.f / 720 + y2 * (1.f / 40320))));
}
CME_DEV bool small_phase(float y) { return fabsf(y) <= 0.5f; }   // false for NaN

// Linear and pump flow of the Strang step, exact, applied as the increment D += e D + c: over
// h/2 (full = false: e = expm1(L h/2), c = (exp(L_0 h/2) - 1)/L_0 sqrt(kappa_ext) A_in on the
// pumped mode) or over h (full = true: e = expm1(L h), c the same over h).
template <typename T, int LOGN, int R, int C>
CME_DEV void strang_linear(const Group<T, LOGN, R, C>& grp, FieldState<T, LOGN, R, C>& fs,
                           const Props<T, LOGN, R, C>& pr, const StepConsts<T>& c, bool full)
{
    constexpr bool COMP = Group<T, LOGN, R, C>::COMP;
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const cx<T> e = full ? pr.get2(j) : pr.get1(j);
        cx<T> d = cmul(e, fs.Dh[j]);
        if constexpr (COMP)
            d = cadd(d, cmul(e, fs.getL(j)));
        if (j == 0 && grp.t == 0)
            d = cadd(d, full ? c.cp2 : c.cp);
        fs.add(j, d);
    }
}

// Exact Kerr flow of the Strang step over h.  With a = inverse transform of D the flow is
// a -> a exp(i g0 |a|^2 h); it is applied as the increment D += DFT(a expm1(i g0 |a|^2 h))/N.
// STORE = true also stores, unless so is null (the adjoint's recomputation), the time-domain
// field a at so[j P] and the state after the flow at so[sstride + j P].
template <bool STORE, typename T, int LOGN, int R, int C>
CME_DEV void strang_kerr(Group<T, LOGN, R, C>& grp, FieldState<T, LOGN, R, C>& fs,
                         const StepConsts<T>& c, cx<T>* so, long long sstride)
{
    constexpr int P = Group<T, LOGN, R, C>::P;
    constexpr T invN = (T)(1.0 / (1 << LOGN));
    cx<T> x[R];
#pragma unroll
    for (int j = 0; j < R; ++j)
        x[j] = fs.Dh[j];
#pragma unroll 1
    for (int d = 0; d < 2; ++d) {
        grp.inverse(x, d);
        if constexpr (STORE) {
            if (d == 0 && so) {
#pragma unroll
                for (int j = 0; j < R; ++j)
                    sstore(so + j * P, x[j]);
            }
        }
        if (d == 0) {
            // expm1(i phi) = (-2 sin^2(phi/2), sin(phi)), phi = g0 |a|^2 h; the forward
            // transform runs as conj(inverse(conj(.))).  FP32: the Taylor series for every
            // value, then sincosf only for values outside its range, behind one branch per
            // thread rather than one per value
            T ph2[R], sn[R], cs[R];
            bool big = false;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                ph2[j] = c.g0h * (x[j].re * x[j].re + x[j].im * x[j].im);
                if constexpr (sizeof(T) == 4) {
                    taylor_sincos(ph2[j], sn[j], cs[j]);
                    big |= !small_phase(ph2[j]);
                } else {
                    sincos(ph2[j], &sn[j], &cs[j]);
                }
            }
            if constexpr (sizeof(T) == 4) {
                if (big) {
#pragma unroll
                    for (int j = 0; j < R; ++j)
                        if (!small_phase(ph2[j]))
                            sincosf(ph2[j], &sn[j], &cs[j]);
                }
            }
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const cx<T> em = {T(-2) * sn[j] * sn[j] * invN, T(2) * sn[j] * cs[j] * invN};
                const cx<T> b = cmul(x[j], em);
                x[j] = {b.re, -b.im};
            }
        }
    }
    grp.mask(x);   // no Kerr increment on padding modes
#pragma unroll
    for (int j = 0; j < R; ++j)
        fs.add(j, cx<T>{x[j].re, -x[j].im});
    if constexpr (STORE) {
        if (so) {
#pragma unroll
            for (int j = 0; j < R; ++j)
                sstore(so + sstride + j * P, fs.Dh[j]);
        }
    }
}

// One Strang split step (Sec. 2 "split-step Fourier method ... field in the frequency domain"):
// exact linear+pump flow over h/2, exact Kerr flow over h, exact linear+pump flow over h/2.
// The adjoint's recomputation takes the steps one by one (STORE: see strang_kerr).
template <bool STORE, typename T, int LOGN, int R, int C>
CME_DEV void strang_step_impl(Group<T, LOGN, R, C>& grp, FieldState<T, LOGN, R, C>& fs,
                              const Props<T, LOGN, R, C>& pr, const StepConsts<T>& c, cx<T>* so,
                              long long sstride)
{
    strang_linear(grp, fs, pr, c, false);
    strang_kerr<STORE>(grp, fs, c, so, sstride);
    strang_linear(grp, fs, pr, c, false);
}

// n Strang steps as the step kernels take them: the half flow that closes a step and the half
// flow that opens the next compose exactly into the flow over h (exp(L h/2)^2 = exp(L h), and
// the pump increments into the increment over h), so the n steps apply n + 1 linear flows
// instead of 2n.  The field after the n steps is that of n single steps up to rounding.
template <typename T, int LOGN, int R, int C>
CME_DEV void strang_steps(Group<T, LOGN, R, C>& grp, FieldState<T, LOGN, R, C>& fs,
                          const Props<T, LOGN, R, C>& pr, const StepConsts<T>& c, long long n)
{
    if (n <= 0)
        return;
    strang_linear(grp, fs, pr, c, false);
    for (long long k = 0; k < n; ++k) {
        strang_kerr<false>(grp, fs, c, static_cast<cx<T>*>(nullptr), 0);
        strang_linear(grp, fs, pr, c, k + 1 < n);
    }
}

template <typename T>
CME_DEV StepConsts<T> step_consts(const StepArgs& a, int inst, int N)
{
    StepConsts<T> c;
    const double2 pd = a.pump[inst];
    c.pump = {(T)pd.x, (T)pd.y};
    const double2 cpd = a.cpump[inst];
    c.cp = {(T)cpd.x, (T)cpd.y};
    const double2 cpd2 = a.cpump2 ? a.cpump2[inst] : make_double2(0.0, 0.0);
    c.cp2 = {(T)cpd2.x, (T)cpd2.y};
    c.gN = (T)(a.g0[inst] / (double)N);
    c.g0h = (T)(a.g0[inst] * a.h * 0.5);
    c.h = Coef<T>::h(a);
    c.hh = Coef<T>::hh(a);
    c.h6 = Coef<T>::h6(a);
    return c;
}

// nsteps steps of the instances [first, first + blockDim.x / P) of the group described by a
// (group-relative indices; groups past a.ninst recompute the last instance and store nothing).
// MASKABLE = false compiles the body without the physical-mode mask (every instance M = N):
// the mask test then folds away at compile time.
template <typename T, int LOGN, int R, int METHOD, bool MASKABLE = true, bool FUSED = false>
CME_DEV void step_body(const StepArgs& a, int first, unsigned char* smem)
{
    using GR = Group<T, LOGN, R>;
    constexpr int N = GR::N, P = GR::P;

    const int g = threadIdx.x / P;
    int inst = first + g;
    const bool valid = inst < a.ninst;
    if (!valid)
        inst = a.ninst - 1;  // duplicate work keeps every group in the barriers; no store
    GR grp;
    grp.setup(smem, g, threadIdx.x - g * P, a.tw);
    const long long off = a.base + (long long)inst * N;
    if constexpr (MASKABLE) {
        if (a.phys)
            grp.set_modes(a.phys[inst]);
        grp.set_kerr(a.kerr, off);
    }
    const int t = grp.t;

    cx<T>* hi = reinterpret_cast<cx<T>*>(a.hi) + off + t;
    cx<T>* lo = reinterpret_cast<cx<T>*>(a.lo) + off + t;
    FieldState<T, LOGN, R> fs;
    fs.bind(grp);
    fs.load(hi, lo);
    const StepConsts<T> c = step_consts<T>(a, inst, N);
    Props<T, LOGN, R> pr;
    pr.init(a, off, t);

    if constexpr (METHOD == METHOD_RK4IP) {
        for (long long n = 0; n < a.nsteps; ++n)
            rk4ip_step<!FUSED && rk_cache_ed<T, LOGN, R, 1>()>(grp, fs, pr, c);
    } else {
        const long long m = a.single_steps ? 1 : a.nsteps;
        for (long long n = 0; n < a.nsteps; n += m)
            strang_steps(grp, fs, pr, c, a.nsteps - n < m ? a.nsteps - n : m);
    }

    bool bad = false;
#pragma unroll
    for (int j = 0; j < R; ++j)
        bad |= !(isfinite(fs.Dh[j].re) && isfinite(fs.Dh[j].im));
    if (valid) {
        fs.store(hi, lo);
        if (bad)
            a.status[inst] = 1;
    }
}

template <typename T, int LOGN, int R, int METHOD, bool MASKABLE>
__global__ void __launch_bounds__(max_threads<LOGN, R>()) step_kernel(const StepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    step_body<T, LOGN, R, METHOD, MASKABLE>(a, blockIdx.x * a.G, smem);
}

// The same steps with each instance spread over a cluster of C blocks (P/C threads each);
// launched with a grid of exactly ninst * C blocks and cluster dimension C, so every block
// holds a real instance and all of them take part in every cluster barrier.
template <typename T, int LOGN, int R, int C, int METHOD>
__global__ void __launch_bounds__(Plan<LOGN, R>::P / C) cluster_step_kernel(const StepArgs a)
{
    using GR = Group<T, LOGN, R, C>;
    constexpr int N = GR::N;
    extern __shared__ __align__(16) unsigned char smem[];
    const int inst = blockIdx.x / C;
    GR grp;
    grp.setup_cluster(smem, cluster_rank(), threadIdx.x, a.tw, a.a2a_fault);
    const long long off = a.base + (long long)inst * N;
    if (a.phys)
        grp.set_modes(a.phys[inst]);
    grp.set_kerr(a.kerr, off);
    const int t = grp.t;

    cx<T>* hi = reinterpret_cast<cx<T>*>(a.hi) + off + t;
    cx<T>* lo = reinterpret_cast<cx<T>*>(a.lo) + off + t;
    FieldState<T, LOGN, R, C> fs;
    fs.bind(grp);
    fs.load(hi, lo);
    const StepConsts<T> c = step_consts<T>(a, inst, N);
    Props<T, LOGN, R, C> pr;
    pr.init(a, off, t);
    cluster_sync();   // every block of the cluster runs before the first remote store

    if constexpr (METHOD == METHOD_RK4IP) {
        for (long long n = 0; n < a.nsteps; ++n)
            rk4ip_step<rk_cache_ed<T, LOGN, R, C>()>(grp, fs, pr, c);
    } else {
        const long long m = a.single_steps ? 1 : a.nsteps;
        for (long long n = 0; n < a.nsteps; n += m)
            strang_steps(grp, fs, pr, c, a.nsteps - n < m ? a.nsteps - n : m);
    }

    bool bad = false;
#pragma unroll
    for (int j = 0; j < R; ++j)
        bad |= !(isfinite(fs.Dh[j].re) && isfinite(fs.Dh[j].im));
    fs.store(hi, lo);
    if (bad)
        a.status[inst] = 1;
    if (grp.failed())
        a.status[inst] = 2;
    cluster_sync();   // no block leaves while a peer may still address its shared memory
}

// Diagnostics: one transform or one right-hand-side evaluation of the current field, written in
// transform order to a.diag_out (same layout as the field).
template <typename T, int LOGN, int R>
__global__ void __launch_bounds__(max_threads<LOGN, R>()) diag_kernel(const StepArgs a)
{
    using GR = Group<T, LOGN, R>;
    constexpr int N = GR::N, P = GR::P;
    extern __shared__ __align__(16) unsigned char smem[];
    const int g = threadIdx.x / P;
    int inst = blockIdx.x * a.G + g;
    const bool valid = inst < a.ninst;
    if (!valid)
        inst = a.ninst - 1;
    GR grp;
    grp.setup(smem, g, threadIdx.x - g * P, a.tw);
    const long long off = a.base + (long long)inst * N;
    if (a.phys)
        grp.set_modes(a.phys[inst]);
    grp.set_kerr(a.kerr, off);
    const int t = grp.t;
    const cx<T>* src = reinterpret_cast<const cx<T>*>(a.hi) + off + t;
    cx<T>* dst = reinterpret_cast<cx<T>*>(a.diag_out) + off + t;
    cx<T> x[R];
#pragma unroll
    for (int j = 0; j < R; ++j)
        x[j] = src[j * P];
    if (a.diag_mode == DIAG_IDFT) {
        GR::TF::template run<+1>(x, grp.tw, grp.buf, grp.par, grp.ad);
    } else if (a.diag_mode == DIAG_DFT) {
        GR::TF::template run<-1>(x, grp.tw, grp.buf, grp.par, grp.ad);
    } else {
        const double2 pd = a.pump[inst];
        grp.rhs(x, (T)(a.g0[inst] / (double)N), cx<T>{(T)pd.x, (T)pd.y});
    }
    if (valid) {
#pragma unroll
        for (int j = 0; j < R; ++j)
            dst[j * P] = x[j];
    }
}

}  // namespace cme
