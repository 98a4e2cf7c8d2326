// Device core of the CME integrator: register/shared-memory Stockham transforms over the mode
// number (Eq. 4), the Kerr term, the pump, and the RK4IP and Strang step bodies (Sec. 2).
//
// Thread mapping.  One instance of N modes is handled by P = N/R threads; thread t holds the
// R field values at transform positions t + j*P (j = 0..R-1) in registers for the whole launch.
// A transform is a sequence of radix-R Stockham passes (the last one may use a smaller radix);
// between passes the group exchanges values through a padded shared-memory buffer.  Both the
// inverse transform (sign +1) and the forward transform (sign -1) start and end with the same
// register assignment, so the Kerr term, the pump and every Runge-Kutta combination are
// register-local.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "cme_internal.h"

#define CME_DEV __device__ __forceinline__
#define CME_HD __host__ __device__

namespace cme {

template <typename T>
struct cx {
    T re, im;
};

template <typename T>
CME_DEV cx<T> cadd(cx<T> a, cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T>
CME_DEV cx<T> csub(cx<T> a, cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T>
CME_DEV cx<T> cmul(cx<T> a, cx<T> b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
// a * conj(b)
template <typename T>
CME_DEV cx<T> cmulc(cx<T> a, cx<T> b) { return {a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im}; }
template <typename T>
CME_DEV cx<T> cscale(cx<T> a, T s) { return {a.re * s, a.im * s}; }
// a + s * b
template <typename T>
CME_DEV cx<T> caxpy(cx<T> a, T s, cx<T> b) { return {a.re + s * b.re, a.im + s * b.im}; }

template <typename T> struct v2;
template <> struct v2<float> { using type = float2; };
template <> struct v2<double> { using type = double2; };

template <typename T>
CME_DEV cx<T> gload(const void* p, long long i)
{
    const typename v2<T>::type v = __ldg(reinterpret_cast<const typename v2<T>::type*>(p) + i);
    return {v.x, v.y};
}
// Store of per-step scratch that is read back only much later (the adjoint's stored steps):
// streaming (evict-first), so that it does not push the batch's tables out of L2.
template <typename T>
CME_DEV void sstore(cx<T>* p, cx<T> v)
{
    using V = typename v2<T>::type;
    V w;
    w.x = v.re;
    w.y = v.im;
    __stcs(reinterpret_cast<V*>(p), w);
}
template <typename T>
CME_DEV cx<T> load(const void* p, long long i)
{
    const typename v2<T>::type v = reinterpret_cast<const typename v2<T>::type*>(p)[i];
    return {v.x, v.y};
}
template <typename T>
CME_DEV void store(void* p, long long i, cx<T> a)
{
    typename v2<T>::type v;
    v.x = a.re;
    v.y = a.im;
    reinterpret_cast<typename v2<T>::type*>(p)[i] = v;
}

// ----------------------------------------------------------------------------------------
// Transform plan: N = 2^LOGN, R values per thread, NS passes, last radix 2^LOG_LAST.
// ----------------------------------------------------------------------------------------
CME_HD constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x >> 1); }

template <int LOGN, int R>
struct Plan {
    static constexpr int N = 1 << LOGN;
    static constexpr int LOGR = ilog2(R);
    static_assert((1 << LOGR) == R && R >= 2 && R <= 16, "radix");
    static_assert(N >= R, "N >= R");
    static constexpr int P = N / R;
    static constexpr int NS = (LOGN + LOGR - 1) / LOGR;
    static constexpr int LOG_LAST = LOGN - (NS - 1) * LOGR;
    CME_HD static constexpr int radix(int s) { return s < NS - 1 ? R : (1 << LOG_LAST); }
    CME_HD static constexpr int L(int s) { return 1 << (s * LOGR); }
    static constexpr int NTW = (NS - 1) * (R - 1);  // register twiddles, stages 1..NS-1
    CME_HD static constexpr int pad(int p) { return p + (p >> 4); }
    static constexpr int BUF = N + N / 16 + 1;      // padded buffer length (elements)
};

// exp(2 pi i k / 16), k = 0..15 (compile-time constants of the in-register DFTs)
CME_DEV constexpr double c16(int k)
{
    constexpr double t[16] = {1.0,
                              0.92387953251128675613,
                              0.70710678118654752440,
                              0.38268343236508977173,
                              0.0,
                              -0.38268343236508977173,
                              -0.70710678118654752440,
                              -0.92387953251128675613,
                              -1.0,
                              -0.92387953251128675613,
                              -0.70710678118654752440,
                              -0.38268343236508977173,
                              0.0,
                              0.38268343236508977173,
                              0.70710678118654752440,
                              0.92387953251128675613};
    return t[k & 15];
}
CME_DEV constexpr double s16(int k) { return c16(k - 4); }

// z * exp(S * 2 pi i k / 16) with the trivial angles done without multiplies.
template <int S, int K, typename T>
CME_DEV cx<T> rot16(cx<T> z)
{
    constexpr int k = ((S > 0 ? K : 16 - K) % 16 + 16) % 16;
    if constexpr (k == 0) {
        return z;
    } else if constexpr (k == 4) {
        return {-z.im, z.re};
    } else if constexpr (k == 8) {
        return {-z.re, -z.im};
    } else if constexpr (k == 12) {
        return {z.im, -z.re};
    } else if constexpr (k == 2 || k == 6 || k == 10 || k == 14) {
        // (+-1 +- i)/sqrt(2)
        constexpr T h = (T)0.70710678118654752440;
        constexpr T cr = (k == 2 || k == 14) ? h : -h;
        constexpr T ci = (k == 2 || k == 6) ? h : -h;
        return {(z.re * (cr > 0 ? 1 : -1) - z.im * (ci > 0 ? 1 : -1)) * h,
                (z.re * (ci > 0 ? 1 : -1) + z.im * (cr > 0 ? 1 : -1)) * h};
    } else {
        constexpr T c = (T)c16(k);
        constexpr T s = (T)s16(k);
        return {z.re * c - z.im * s, z.re * s + z.im * c};
    }
}

CME_HD constexpr int bitrev(int x, int bits)
{
    int r = 0;
    for (int i = 0; i < bits; ++i)
        if (x & (1 << i))
            r |= 1 << (bits - 1 - i);
    return r;
}

// In-register DFT of size r (natural order in and out): v[k] = sum_j v[j] exp(S 2 pi i jk/r).
// Radix-2 decimation in frequency; the bit reversal at the end is a register renaming.
template <int r, int S, int span, typename T>
CME_DEV void dft_stage(cx<T> (&v)[r])
{
    if constexpr (span >= 1) {
#pragma unroll
        for (int blk = 0; blk < r; blk += 2 * span) {
#pragma unroll
            for (int j = 0; j < span; ++j) {
                const cx<T> a = v[blk + j], b = v[blk + j + span];
                v[blk + j] = cadd(a, b);
                v[blk + j + span] = csub(a, b);
            }
        }
        // twiddles exp(S 2 pi i j / (2 span)) on the lower halves
#pragma unroll
        for (int blk = 0; blk < r; blk += 2 * span) {
            if constexpr (span >= 2) {
                v[blk + span + 1] = rot16<S, 16 / (2 * span) * 1>(v[blk + span + 1]);
            }
            if constexpr (span >= 4) {
                v[blk + span + 2] = rot16<S, 16 / (2 * span) * 2>(v[blk + span + 2]);
                v[blk + span + 3] = rot16<S, 16 / (2 * span) * 3>(v[blk + span + 3]);
            }
            if constexpr (span >= 8) {
                v[blk + span + 4] = rot16<S, 4>(v[blk + span + 4]);
                v[blk + span + 5] = rot16<S, 5>(v[blk + span + 5]);
                v[blk + span + 6] = rot16<S, 6>(v[blk + span + 6]);
                v[blk + span + 7] = rot16<S, 7>(v[blk + span + 7]);
            }
        }
        dft_stage<r, S, span / 2>(v);
    }
}

template <int r, int S, typename T>
CME_DEV void dft(cx<T> (&v)[r])
{
    static_assert(r <= 16, "in-register DFT up to 16");
    if constexpr (r > 1) {
        dft_stage<r, S, r / 2>(v);
        cx<T> t[r];
#pragma unroll
        for (int k = 0; k < r; ++k)
            t[k] = v[bitrev(k, ilog2(r))];
#pragma unroll
        for (int k = 0; k < r; ++k)
            v[k] = t[k];
    }
}

// ----------------------------------------------------------------------------------------
// Thread-block clusters: one instance spread over C blocks of a cluster, exchanging through
// distributed shared memory (stores into the peer block's shared memory, then a cluster
// barrier whose release/acquire makes them visible).
// ----------------------------------------------------------------------------------------
CME_DEV uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// address of the same shared-memory offset in block `rank` of this cluster
CME_DEV uint32_t dsmem_map(uint32_t a, int rank)
{
    uint32_t r;
    asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
CME_DEV void dsmem_put(uint32_t a, float re, float im)
{
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(re), "f"(im) : "memory");
}
CME_DEV void dsmem_put(uint32_t a, double v)
{
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}
// Asynchronous store into a peer block's shared memory whose completion (its byte count) is
// signalled on an mbarrier in the receiving block (both shared::cluster addresses).
CME_DEV void dsmem_put_async(uint32_t a, float re, float im, uint32_t mbar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];"
                 ::"r"(a), "f"(re), "f"(im), "r"(mbar) : "memory");
}
CME_DEV void dsmem_put_async(uint32_t a, double v, uint32_t mbar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f64 [%0], %1, [%2];"
                 ::"r"(a), "d"(v), "r"(mbar) : "memory");
}
CME_DEV void mbar_init(uint32_t mb, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(count) : "memory");
}
// make the initialisation of this block's mbarriers visible to the cluster's other blocks
CME_DEV void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// one arrival that also expects `bytes` more bytes of asynchronous stores in this phase
CME_DEV void mbar_arrive_expect_tx(uint32_t mb, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes)
                 : "memory");
}
// has the phase of parity `parity` completed?
CME_DEV bool mbar_try_wait(uint32_t mb, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(mb), "r"(parity) : "memory");
    return ok != 0;
}
// Bounded wait: at most `tries` polls (each may suspend the thread briefly); false if the
// phase did not complete.
CME_DEV bool mbar_wait(uint32_t mb, uint32_t parity, int tries)
{
    for (int k = 0; k < tries; ++k)
        if (mbar_try_wait(mb, parity))
            return true;
    return false;
}
// Bulk asynchronous copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from
// global memory into this block's shared memory, its completion counted on mbarrier `mbar`.
CME_DEV void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"((unsigned long long)__cvta_generic_to_global(src)), "r"(bytes),
                 "r"(mbar) : "memory");
}
// order this thread's earlier generic-proxy accesses of shared memory before its later
// asynchronous-proxy writes (bulk copies) into it
CME_DEV void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
CME_DEV void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
CME_DEV int cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return (int)r;
}

// ----------------------------------------------------------------------------------------
// Shared-memory exchange buffer: float2 words for FP32, separate re/im arrays for FP64 (so
// both are 8-byte accesses with the same bank pattern).
// ----------------------------------------------------------------------------------------
template <typename T> struct Xbuf;
template <>
struct Xbuf<float> {
    float2* p;
    CME_DEV void put(int i, cx<float> v) const { p[i] = make_float2(v.re, v.im); }
    CME_DEV cx<float> get(int i) const
    {
        const float2 a = p[i];
        return {a.x, a.y};
    }
    CME_DEV Xbuf at(int off) const { return {p + off}; }
    // element at DSMEM address a (a maps element i of some block's buffer)
    CME_DEV void put_remote(uint32_t a, cx<float> v) const { dsmem_put(a, v.re, v.im); }
    CME_DEV void put_remote_async(uint32_t a, cx<float> v, uint32_t mbar) const
    {
        dsmem_put_async(a, v.re, v.im, mbar);
    }
    static constexpr int words_per_elem = 1;  // in 8-byte words
};
template <>
struct Xbuf<double> {
    double* re;  // im = re + BUF
    int stride;
    CME_DEV void put(int i, cx<double> v) const
    {
        re[i] = v.re;
        re[i + stride] = v.im;
    }
    CME_DEV cx<double> get(int i) const { return {re[i], re[i + stride]}; }
    CME_DEV Xbuf at(int off) const { return {re + 2 * off, stride}; }
    CME_DEV void put_remote(uint32_t a, cx<double> v) const
    {
        dsmem_put(a, v.re);
        dsmem_put(a + 8u * (uint32_t)stride, v.im);
    }
    CME_DEV void put_remote_async(uint32_t a, cx<double> v, uint32_t mbar) const
    {
        dsmem_put_async(a, v.re, mbar);
        dsmem_put_async(a + 8u * (uint32_t)stride, v.im, mbar);
    }
    static constexpr int words_per_elem = 2;
};

template <bool WARP>
CME_DEV void group_sync()
{
    if constexpr (WARP)
        __syncwarp();
    else
        __syncthreads();
}


// ----------------------------------------------------------------------------------------
// Transform of one group: x holds positions t + j*P; sign S (+1 inverse / time samples,
// -1 forward).  tw holds exp(+2 pi i j k/(L r)) for the passes s >= 1.
// ----------------------------------------------------------------------------------------
template <typename T, int LOGN, int R, bool WARP>
struct Transform {
    using PL = Plan<LOGN, R>;
    static constexpr int N = PL::N, P = PL::P, NS = PL::NS;
    static constexpr int BUF = PL::BUF;   // elements per exchange buffer

    template <int s, int S, class TW>
    CME_DEV static void pass(cx<T> (&x)[R], const TW& tw)
    {
        constexpr int r = PL::radix(s), Q = R / r;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            cx<T> v[r];
#pragma unroll
            for (int j = 0; j < r; ++j)
                v[j] = x[q + j * Q];
            if constexpr (s > 0) {
#pragma unroll
                for (int j = 1; j < r; ++j) {
                    const cx<T> w = tw.template get<s>(q, j);
                    v[j] = (S > 0) ? cmul(v[j], w) : cmulc(v[j], w);
                }
            }
            dft<r, S>(v);
#pragma unroll
            for (int j = 0; j < r; ++j)
                x[q + j * Q] = v[j];
        }
    }

    // Per-thread shared-memory addressing, computed once per launch.  With the padding
    // p -> p + (p >> 4) every exchange address is a per-thread base plus a compile-time
    // offset: for the write of pass s (radix R, stride L = R^s) the thread's base is
    // b = (t - k) R + k, k = t mod L, and (b mod 16) + (jL mod 16) < 16 for all j < R, so
    // pad(b + jL) = pad(b) + jL + (jL >> 4); likewise pad(t + jP) = pad(t) + jP + (jP >> 4)
    // (both checked by enumeration for every compiled N and R = 2 ... 16).
    struct Addr {
        int rd;
        int wr[NS > 1 ? NS - 1 : 1];
        int wx0, wx1, rx0, rx1;   // XOR-layout bases of the stride-8 exchange (R = 8)
    };
    // The exchange after a radix-8 pass of stride L = 8 uses the XOR layout
    // p -> p ^ (8 * bit6(p)) instead of the padding: its writes (p = 64 (t >> 3) + (t & 7) + 8j)
    // and reads (p = t + jP) then hit 16 distinct 8-byte banks per half-warp, and every address
    // is one of two per-thread bases plus a compile-time offset.
    CME_HD static constexpr bool xor8(int s) { return R == 8 && PL::L(s) == 8 && P >= 16; }

    CME_DEV static Addr make_addr(int t)
    {
        Addr a;
        a.rd = PL::pad(t);
#pragma unroll
        for (int s = 0; s + 1 < NS; ++s) {
            const int L = PL::L(s);
            const int k = t & (L - 1);
            a.wr[s] = PL::pad((t - k) * R + k);
        }
        // stride-8 exchange: write base 64 (t >> 3) + (t & 7), flipped by 8 c, c = bit 3 of t
        const int c = (t >> 3) & 1;
        const int wb = 64 * (t >> 3) + (t & 7);
        a.wx0 = wb + 8 * c;       // even j
        a.wx1 = wb - 8 * c;       // odd j
        a.rx0 = t ^ (8 * ((t >> 6) & 1));
        a.rx1 = a.rx0 ^ 8;        // reads whose jP has bit 6 set
        return a;
    }

    template <int s>
    CME_DEV static void exchange(cx<T> (&x)[R], const Xbuf<T>& b, const Addr& ad, int par)
    {
        static_assert(PL::radix(s) == R, "exchanges follow full-radix passes");
        constexpr int L = PL::L(s);
        const Xbuf<T> mine = b.at(par * BUF);
        if constexpr (xor8(s)) {
#pragma unroll
            for (int j = 0; j < R; ++j)
                mine.put(((j & 1) ? ad.wx1 : ad.wx0) + 8 * j, x[j]);
            group_sync<WARP>();
#pragma unroll
            for (int j = 0; j < R; ++j)
                x[j] = mine.get((((j * P) >> 6) & 1 ? ad.rx1 : ad.rx0) + j * P);
        } else {
#pragma unroll
            for (int j = 0; j < R; ++j)
                mine.put(ad.wr[s] + j * L + ((j * L) >> 4), x[j]);
            group_sync<WARP>();
#pragma unroll
            for (int j = 0; j < R; ++j)
                x[j] = mine.get(ad.rd + j * P + ((j * P) >> 4));
        }
    }

    // buf: the first of two ping-pong buffers (the second starts BUF elements later); par
    // selects the one the next exchange writes.
    template <int s, int S, class TW>
    CME_DEV static void run_from(cx<T> (&x)[R], const TW& tw, const Xbuf<T>& buf, int& par,
                                 const Addr& ad)
    {
        pass<s, S>(x, tw);
        if constexpr (s + 1 < NS) {
            exchange<s>(x, buf, ad, par);
            par ^= 1;
            run_from<s + 1, S, TW>(x, tw, buf, par, ad);
        }
    }

    template <int S, class TW>
    CME_DEV static void run(cx<T> (&x)[R], const TW& tw, const Xbuf<T>& buf, int& par,
                            const Addr& ad)
    {
        run_from<0, S, TW>(x, tw, buf, par, ad);
    }
};

// ----------------------------------------------------------------------------------------
// Four-step transform of one instance spread over the C blocks of a thread-block cluster
// (N = C N2, P = N/R threads in all, PC = P/C per block; C divides R, G = R/C).
//
// With k = k1 + C k2 (k1 < C, k2 < N2) and n = n2 + N2 n1 (n2 < N2, n1 < C),
//   a_n = sum_k1 exp(2 pi i n1 k1 / C) exp(2 pi i n2 k1 / N) sum_k2 X_k exp(2 pi i n2 k2 / N2),
// so the inverse transform is an N2-point transform inside each block (block r holds k1 = r),
// a twiddle, one all-to-all between the blocks, and C-point transforms in registers.
//   Modes: thread l of block r holds k = r + C (l + PC j) = t + jP with t = r + C l.
//   Time samples: the same thread holds n = t' + jP with t' = r PC + l.
// Both layouts have the form t + jP, so the pointwise work (Kerr term, pump, Runge-Kutta
// algebra, loads and stores) is unchanged; only which thread holds which mode differs.  The
// transform from time samples back to modes runs the same stages in reverse order (the
// forward transform is conj(inverse(conj .)) as for one block).
//
// One all-to-all moves every value once: each thread stores its R values into C blocks'
// buffers with asynchronous stores, consecutive threads writing consecutive words, and each
// store counts its bytes on an mbarrier of the receiving block; a block's threads wait for
// that mbarrier's phase (all N2 values of its buffer arrived) instead of a cluster barrier.
// Two ping-pong buffers per block, each with its own mbarrier.  A buffer is written again two
// all-to-alls later, and that cannot start before every thread of the receiving block has
// read it: a sender first needs the receiving block's next all-to-all values, and each
// thread's stores there depend on the values it read (every thread stores into every block).
// ----------------------------------------------------------------------------------------
template <typename T, int LOGN, int R, int C>
struct ClusterFFT {
    static constexpr int LC = ilog2(C);
    static_assert((1 << LC) == C && C >= 2 && C <= R && R % C == 0, "C divides R");
    static constexpr int N = 1 << LOGN, P = N / R, PC = P / C, N2 = N / C, G = R / C;
    static constexpr bool WARP = PC <= 32;
    using TL = Transform<T, LOGN - LC, R, WARP>;     // the N2-point transform of one block
    static_assert(TL::P == PC, "block threads");

    // In-register C-point inverse transforms over slots {c G + m : c < C}, m < G.
    CME_DEV static void radix_c(cx<T> (&x)[R])
    {
#pragma unroll
        for (int m = 0; m < G; ++m) {
            cx<T> v[C];
#pragma unroll
            for (int c = 0; c < C; ++c)
                v[c] = x[c * G + m];
            dft<C, +1>(v);
#pragma unroll
            for (int c = 0; c < C; ++c)
                x[c * G + m] = v[c];
        }
    }
};

// Twiddles exp(2 pi i j k / (L r)) of pass s >= 1 for butterfly q of thread t, where
// k = (t + qP) mod L, taken from the table exp(2 pi i m / N).  IN_REGS = true loads all of
// them into registers once per launch; otherwise each pass reads them from the table through
// the read-only cache (large N, where registers are scarce).
// TS: the table holds exp(2 pi i m / (TS N)) (a larger transform's table, read at stride TS).
template <typename T, int LOGN, int R, bool IN_REGS, int TS = 1>
struct Twiddles;

template <typename T, int LOGN, int R, int TS>
struct Twiddles<T, LOGN, R, true, TS> {
    using PL = Plan<LOGN, R>;
    cx<T> w[PL::NTW > 0 ? PL::NTW : 1];

    template <int s>
    CME_DEV void init_from(const void* table, int t)
    {
        if constexpr (s < PL::NS) {
            constexpr int r = PL::radix(s), Q = R / r, L = PL::L(s);
            constexpr int stride = PL::N / (L * r);
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int k = (t + q * PL::P) & (L - 1);
#pragma unroll
                for (int j = 1; j < r; ++j)
                    w[(s - 1) * (R - 1) + q * (r - 1) + (j - 1)] =
                        gload<T>(table, ((j * k * stride) & (PL::N - 1)) * TS);
            }
            init_from<s + 1>(table, t);
        }
    }
    CME_DEV void init(const void* table, int t)
    {
        if constexpr (PL::NS > 1)
            init_from<1>(table, t);
    }
    template <int s>
    CME_DEV cx<T> get(int q, int j) const
    {
        constexpr int r = PL::radix(s);
        return w[(s - 1) * (R - 1) + q * (r - 1) + (j - 1)];
    }
};

template <typename T, int LOGN, int R, int TS>
struct Twiddles<T, LOGN, R, false, TS> {
    using PL = Plan<LOGN, R>;
    const cx<T>* table;
    int kst[PL::NS > 1 ? PL::NS : 1];  // (t mod L_s) * N / (L_s r_s) per pass

    CME_DEV void init(const void* tbl, int t)
    {
        table = reinterpret_cast<const cx<T>*>(tbl);
#pragma unroll
        for (int s = 1; s < PL::NS; ++s) {
            const int L = PL::L(s), r = PL::radix(s);
            kst[s] = (t & (L - 1)) * (PL::N / (L * r));
        }
    }
    template <int s>
    CME_DEV cx<T> get(int q, int j) const
    {
        // butterfly q > 0 only occurs in the last pass, where k = t + qP exactly
        constexpr int r = PL::radix(s), L = PL::L(s), stride = PL::N / (L * r);
        return gload<T>(table, ((j * kst[s] + j * q * PL::P * stride) & (PL::N - 1)) * TS);
    }
};

// The same twiddles held in shared memory, each thread's in its own slots of a thread-major
// array [(pass, butterfly, j)][P] (no bank conflicts; no thread reads another's slot, so no
// barrier is needed after the fill).  Used where registers are too scarce and the table loads
// would crowd the global-load queue (FP32, N >= 2048).
template <typename T, int LOGN, int R, int TS = 1>
struct TwiddlesSmem {
    using PL = Plan<LOGN, R>;
    const cx<T>* base;   // this thread's slot 0

    CME_DEV void init(const void* table, int t, cx<T>* smem_tw)
    {
        base = smem_tw + t;
        init_from<1>(table, t, smem_tw);
    }
    template <int s>
    CME_DEV void init_from(const void* table, int t, cx<T>* smem_tw)
    {
        if constexpr (s < PL::NS) {
            constexpr int r = PL::radix(s), Q = R / r, L = PL::L(s);
            constexpr int stride = PL::N / (L * r);
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int k = (t + q * PL::P) & (L - 1);
#pragma unroll
                for (int j = 1; j < r; ++j)
                    smem_tw[((s - 1) * (R - 1) + q * (r - 1) + (j - 1)) * PL::P + t] =
                        gload<T>(table, ((j * k * stride) & (PL::N - 1)) * TS);
            }
            init_from<s + 1>(table, t, smem_tw);
        }
    }
    template <int s>
    CME_DEV cx<T> get(int q, int j) const
    {
        constexpr int r = PL::radix(s);
        return base[((s - 1) * (R - 1) + q * (r - 1) + (j - 1)) * PL::P];
    }
};

// Compensated update (hi, lo) += d with an exact two-sum of hi and (lo + d).
template <typename T, bool COMP>
CME_DEV void accumulate(cx<T>& hi, cx<T>& lo, cx<T> d)
{
    if constexpr (COMP) {
        const T yr = lo.re + d.re, yi = lo.im + d.im;
        const T sr = hi.re + yr, si = hi.im + yi;
        const T br = sr - hi.re, bi = si - hi.im;
        lo.re = (hi.re - (sr - br)) + (yr - br);
        lo.im = (hi.im - (si - bi)) + (yi - bi);
        hi.re = sr;
        hi.im = si;
    } else {
        hi.re += d.re;
        hi.im += d.im;
    }
}

}  // namespace cme
