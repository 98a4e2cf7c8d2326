// Persistent step kernels: one launch advances every instance of a uniform-N group by nsteps
// RK4IP or Strang steps with the field held in registers throughout.
#pragma once

#include "cme_core.cuh"

namespace cme {

// Per-thread view of one instance: the transform machinery plus the instance constants.
template <typename T, int LOGN, int R>
struct Group {
    using PL = Plan<LOGN, R>;
    static constexpr int N = PL::N, P = PL::P;
    static constexpr bool WARP = (P <= 32);
    static constexpr bool COMP = (sizeof(T) == 4);  // compensated state in FP32
    using TF = Transform<T, LOGN, R, WARP>;

    int t;
    int par;
    Xbuf<T> buf[2];
    cx<T> tw[PL::NTW > 0 ? PL::NTW : 1];

    // F(x) = pump + i (g0/N) DFT(|a|^2 a), a = inverse transform of x   (Eq. 4)
    CME_DEV void rhs(cx<T> (&x)[R], T gN, cx<T> pump)
    {
        TF::template run<+1>(x, tw, buf, par, t);
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const T c = gN * (x[j].re * x[j].re + x[j].im * x[j].im);
            x[j] = {-c * x[j].im, c * x[j].re};
        }
        TF::template run<-1>(x, tw, buf, par, t);
        if (t == 0)
            x[0] = cadd(x[0], pump);
    }
};

// Set up the shared-memory exchange buffers of group g.
template <typename T, int LOGN, int R>
CME_DEV void setup_buffers(Group<T, LOGN, R>& grp, unsigned char* smem, int g)
{
    using PL = Plan<LOGN, R>;
    constexpr int W = Xbuf<T>::words_per_elem;  // 8-byte words per element
    constexpr int BUF = PL::BUF;
    double* base = reinterpret_cast<double*>(smem) + (size_t)g * 2 * W * BUF;
    if constexpr (sizeof(T) == 4) {
        grp.buf[0].p = reinterpret_cast<float2*>(base);
        grp.buf[1].p = reinterpret_cast<float2*>(base + BUF);
    } else {
        grp.buf[0].re = base;
        grp.buf[0].im = base + BUF;
        grp.buf[1].re = base + 2 * BUF;
        grp.buf[1].im = base + 3 * BUF;
    }
}

template <typename T, int LOGN, int R, int METHOD>
__global__ void __launch_bounds__((Plan<LOGN, R>::P > 256 ? Plan<LOGN, R>::P : 256))
    step_kernel(const StepArgs a)
{
    using GR = Group<T, LOGN, R>;
    constexpr int N = GR::N, P = GR::P;
    constexpr bool COMP = GR::COMP;
    extern __shared__ __align__(16) unsigned char smem[];

    const int g = threadIdx.x / P;
    GR grp;
    grp.t = threadIdx.x - g * P;
    grp.par = 0;
    int inst = blockIdx.x * a.G + g;
    const bool valid = inst < a.ninst;
    if (!valid)
        inst = a.ninst - 1;  // duplicate work keeps every group in the barriers; no store
    setup_buffers<T, LOGN, R>(grp, smem, g);
    GR::TF::load_tw(grp.tw, a.tw, grp.t);

    const long long off = a.base + (long long)inst * N;
    const int t = grp.t;
    cx<T> Dh[R], Dl[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        Dh[j] = load<T>(a.hi, off + t + j * P);
        if constexpr (COMP)
            Dl[j] = load<T>(a.lo, off + t + j * P);
        else
            Dl[j] = {T(0), T(0)};
    }
    const double2 pd = a.pump[inst];
    const cx<T> pump = {(T)pd.x, (T)pd.y};
    const T gN = (T)(a.g0[inst] / (double)N);
    const T h = (T)a.h, hh = (T)(0.5 * a.h), h6 = (T)(a.h / 6.0);

    if constexpr (METHOD == METHOD_RK4IP) {
        // RK4IP (Sec. 2 "fourth-order Runge-Kutta"; Hult 2007) written as increments of D:
        //   x2 = D + (e1 D + h/2 k1),  x3 = D + (e1 D + h/2 k2),  x4 = D + (e2 D + h E k3),
        //   D' = D + e2 D + h/6 [E (k1 + 2 k2 + 2 k3) + k4],  k1 = E F(D),  k_i = F(x_i),
        // with E = exp(L h/2), e1 = expm1(L h/2), e2 = expm1(L h).
        for (long long n = 0; n < a.nsteps; ++n) {
            cx<T> x[R], S[R];
#pragma unroll
            for (int j = 0; j < R; ++j)
                x[j] = Dh[j];
            grp.rhs(x, gN, pump);
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const long long m = off + t + j * P;
                const cx<T> E = gload<T>(a.E, m), e1 = gload<T>(a.e1, m);
                const cx<T> k1 = cmul(E, x[j]);
                S[j] = cmul(E, k1);
                x[j] = cadd(Dh[j], caxpy(cmul(e1, Dh[j]), hh, k1));
            }
            grp.rhs(x, gN, pump);
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const long long m = off + t + j * P;
                const cx<T> E = gload<T>(a.E, m), e1 = gload<T>(a.e1, m);
                S[j] = caxpy(S[j], T(2), cmul(E, x[j]));
                x[j] = cadd(Dh[j], caxpy(cmul(e1, Dh[j]), hh, x[j]));
            }
            grp.rhs(x, gN, pump);
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const long long m = off + t + j * P;
                const cx<T> E = gload<T>(a.E, m), e2 = gload<T>(a.e2, m);
                const cx<T> Ek3 = cmul(E, x[j]);
                S[j] = caxpy(S[j], T(2), Ek3);
                x[j] = cadd(Dh[j], caxpy(cmul(e2, Dh[j]), h, Ek3));
            }
            grp.rhs(x, gN, pump);
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const long long m = off + t + j * P;
                const cx<T> e2 = gload<T>(a.e2, m);
                cx<T> d = cmul(e2, Dh[j]);
                if constexpr (COMP)
                    d = cadd(d, cmul(e2, Dl[j]));
                d = caxpy(d, h6, cadd(S[j], x[j]));
                accumulate<T, COMP>(Dh[j], Dl[j], d);
            }
        }
    } else {
        // Strang split step (Sec. 2 "split-step Fourier method ... field in the frequency
        // domain"): exact linear+pump flow over h/2, exact Kerr flow over h, exact linear+pump
        // flow over h/2.  With a = inverse transform of D the Kerr flow is
        // a -> a exp(i g0 |a|^2 h); it is applied as the increment D += DFT(a expm1(...))/N.
        const double2 cpd = a.cpump[inst];
        const cx<T> cp = {(T)cpd.x, (T)cpd.y};
        const T g0h = (T)(a.g0[inst] * a.h * 0.5);   // half Kerr phase per |a|^2
        const T invN = (T)(1.0 / N);
        for (long long n = 0; n < a.nsteps; ++n) {
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                if (half == 1) {
                    cx<T> x[R];
#pragma unroll
                    for (int j = 0; j < R; ++j)
                        x[j] = Dh[j];
                    GR::TF::template run<+1>(x, grp.tw, grp.buf, grp.par, t);
#pragma unroll
                    for (int j = 0; j < R; ++j) {
                        // expm1(i phi) = (-2 sin^2(phi/2), sin(phi)), phi = g0 |a|^2 h
                        const T ph2 = g0h * (x[j].re * x[j].re + x[j].im * x[j].im);
                        T s, c;
                        if constexpr (sizeof(T) == 4)
                            sincosf(ph2, &s, &c);
                        else
                            sincos(ph2, &s, &c);
                        const cx<T> em = {T(-2) * s * s * invN, T(2) * s * c * invN};
                        x[j] = cmul(x[j], em);
                    }
                    GR::TF::template run<-1>(x, grp.tw, grp.buf, grp.par, t);
#pragma unroll
                    for (int j = 0; j < R; ++j)
                        accumulate<T, COMP>(Dh[j], Dl[j], x[j]);
                }
                // linear + pump half step: D += e1 D + delta_{mu,0} c
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    const long long m = off + t + j * P;
                    const cx<T> e1 = gload<T>(a.e1, m);
                    cx<T> d = cmul(e1, Dh[j]);
                    if constexpr (COMP)
                        d = cadd(d, cmul(e1, Dl[j]));
                    if (j == 0 && t == 0)
                        d = cadd(d, cp);
                    accumulate<T, COMP>(Dh[j], Dl[j], d);
                }
            }
        }
    }

    bool bad = false;
#pragma unroll
    for (int j = 0; j < R; ++j)
        bad |= !(isfinite(Dh[j].re) && isfinite(Dh[j].im));
    if (valid) {
#pragma unroll
        for (int j = 0; j < R; ++j) {
            store<T>(a.hi, off + t + j * P, Dh[j]);
            if constexpr (COMP)
                store<T>(a.lo, off + t + j * P, Dl[j]);
        }
        if (bad)
            a.status[inst] = 1;
    }
}

// Diagnostics: one transform or one right-hand-side evaluation of the current field, written in
// transform order to a.diag_out (same layout as the field).
template <typename T, int LOGN, int R>
__global__ void __launch_bounds__((Plan<LOGN, R>::P > 256 ? Plan<LOGN, R>::P : 256))
    diag_kernel(const StepArgs a)
{
    using GR = Group<T, LOGN, R>;
    constexpr int N = GR::N, P = GR::P;
    extern __shared__ __align__(16) unsigned char smem[];
    const int g = threadIdx.x / P;
    GR grp;
    grp.t = threadIdx.x - g * P;
    grp.par = 0;
    int inst = blockIdx.x * a.G + g;
    const bool valid = inst < a.ninst;
    if (!valid)
        inst = a.ninst - 1;
    setup_buffers<T, LOGN, R>(grp, smem, g);
    GR::TF::load_tw(grp.tw, a.tw, grp.t);
    const long long off = a.base + (long long)inst * N;
    const int t = grp.t;
    cx<T> x[R];
#pragma unroll
    for (int j = 0; j < R; ++j)
        x[j] = load<T>(a.hi, off + t + j * P);
    if (a.diag_mode == DIAG_IDFT) {
        GR::TF::template run<+1>(x, grp.tw, grp.buf, grp.par, t);
    } else if (a.diag_mode == DIAG_DFT) {
        GR::TF::template run<-1>(x, grp.tw, grp.buf, grp.par, t);
    } else {
        const double2 pd = a.pump[inst];
        grp.rhs(x, (T)(a.g0[inst] / (double)N), cx<T>{(T)pd.x, (T)pd.y});
    }
    if (valid) {
#pragma unroll
        for (int j = 0; j < R; ++j)
            store<T>(a.diag_out, off + t + j * P, x[j]);
    }
}

}  // namespace cme
