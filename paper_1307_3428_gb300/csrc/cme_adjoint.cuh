// Discrete adjoint of the RK4IP step kernels (reverse mode through exactly the forward
// algebra) for gradients of a loss on the final field with respect to the initial field, the
// linear operator L_mu = -kappa_mu/2 + i(omega_mu - omega_0 - sigma) and the pump.
//
// Cotangents of complex quantities follow vbar = dL/dRe v + i dL/dIm v, so that for y = a x
// xbar += conj(a) ybar and abar += conj(x) ybar.  The right-hand side F(x) = pump +
// i g0/N DFT(|a|^2 a), a = IDFT(x), has the vector-Jacobian product
//     bbar = IDFT(-i g0 ybar) / N,   abar = 2 |a|^2 bbar + a^2 conj(bbar),   xbar = DFT(abar),
// evaluated with the same transform code as the forward pass.
//
// Memory and schedule: the forward pass stores the field at the start of every segment of K
// steps (checkpoints).  The backward pass then walks the segments in reverse.  For each segment
// s, a recompute kernel regenerates, from its checkpoint, the state D, the stage values
// y1 = F(D), k2, k3 and the time-domain fields a = IDFT(stage input) of the four stages of
// every step into one half of a two-segment buffer.  A backward kernel then runs the four
// vector-Jacobian products of every step of s from that half (two transforms each, since a
// comes from the buffer).  The
// recomputation of segment s - 1 does not depend on any cotangent, so the host runs it on a
// second stream while segment s runs backwards: only the products are on the critical path.
#pragma once

#include "cme_adjoint_args.h"
#include "cme_step.cuh"

namespace cme {

template <typename T>
CME_DEV cx<T> cconj(cx<T> a) { return {a.re, -a.im}; }

// Accumulator of one mode's L cotangent over the steps of a segment; the running total lives in
// FP64 in memory between segments.  FP64 kernels continue the total term by term (so the sum,
// and the gradient, do not depend on the segment length).  FP32 kernels keep the segment's
// terms in a compensated float pair and add it to the total once per
// segment: FP64 arithmetic runs at 1/64 of the FP32 rate on this GPU, and a convert-and-add
// per term made it the bottleneck of the backward pass.  The pair is a Kahan sum (4 adds per
// term, against 7 for an exact two-sum, on the backward pass's dependency chains).
template <typename T>
struct LAcc;
template <>
struct LAcc<double> {
    double2 v;
    CME_DEV void init(double2 total) { v = total; }
    CME_DEV void add(cx<double> d)
    {
        v.x += d.re;
        v.y += d.im;
    }
    CME_DEV double2 finish(double2) const { return v; }
};
template <>
struct LAcc<float> {
    float hr, hi, cr, ci;   // running sums and their Kahan compensations (minus the lost parts)
    CME_DEV void init(double2) { hr = hi = cr = ci = 0.f; }
    CME_DEV static void kahan(float& h, float& c, float d)
    {
        const float y = d - c, t = h + y;
        c = (t - h) - y;
        h = t;
    }
    CME_DEV void add(cx<float> d)
    {
        kahan(hr, cr, d.re);
        kahan(hi, ci, d.im);
    }
    CME_DEV double2 finish(double2 total) const
    {
        return make_double2(total.x + ((double)hr - (double)cr), total.y + ((double)hi - (double)ci));
    }
};

// Per-instance set-up shared by both roles.  C > 1: each instance is spread over a cluster of
// C blocks (grid = ninst * C blocks of P/C threads, cluster dimension C).
template <typename T, int LOGN, int R, int C>
CME_DEV int adj_setup(Group<T, LOGN, R, C>& grp, unsigned char* smem, const StepArgs& a,
                      bool& valid)
{
    constexpr int P = Group<T, LOGN, R, C>::P;
    int inst;
    valid = true;
    if constexpr (C == 1) {
        const int g = threadIdx.x / P;
        inst = blockIdx.x * a.G + g;
        valid = inst < a.ninst;
        if (!valid)
            inst = a.ninst - 1;
        grp.setup(smem, g, threadIdx.x - g * P, a.tw);
    } else {
        inst = blockIdx.x / C;
        grp.setup_cluster(smem, cluster_rank(), threadIdx.x, a.tw, a.a2a_fault);
    }
    if (a.phys)
        grp.set_modes(a.phys[inst]);
    grp.set_kerr(a.kerr, a.base + (long long)inst * Group<T, LOGN, R, C>::N);
    return inst;
}

template <int LOGN, int R, int C>
constexpr int adj_threads() { return C == 1 ? max_threads<LOGN, R>() : Plan<LOGN, R>::P / C; }

// FP32 backward kernels of cluster groups prefetch the stored data of the next step (ADJ_VECS
// vectors, R chunks of P/C values each per block) into shared memory with bulk asynchronous
// copies while they process the current one, where two steps' worth fits beside the cluster
// transform's buffers (N = 4096 x 16 gradient: 219 -> 188 ms).  FP64 gradients run their
// recomputation and backward blocks on shared SMs (8-block clusters), which the larger
// block would no longer allow (2.4e8 -> 1.4e8 gradient mode-steps/s), and FP64 steps are
// bound by the FP64 pipes, not by these loads.
template <typename T, int LOGN, int R, int C>
CME_HD constexpr size_t adj_prefetch_bytes()
{
    return C > 1 ? (size_t)2 * ADJ_VECS * R * (Plan<LOGN, R>::P / C) * sizeof(cx<T>) : 0;
}
template <typename T, int LOGN, int R, int C>
CME_HD constexpr bool adj_prefetch()
{
    if constexpr (C == 1 || sizeof(T) != 4)
        return false;
    else
        return cluster_smem_bytes<T, LOGN, R, C>() + adj_prefetch_bytes<T, LOGN, R, C>() + 16 <=
               (size_t)200 * 1024;
}
// dynamic shared memory of the backward kernel of a cluster group
template <typename T, int LOGN, int R, int C>
CME_HD constexpr size_t adj_backward_smem()
{
    return cluster_smem_bytes<T, LOGN, R, C>() +
           (adj_prefetch<T, LOGN, R, C>() ? adj_prefetch_bytes<T, LOGN, R, C>() + 16 : 0);
}

// Recompute role: the states of segment A.seg from checkpoint A.ckpt_slot and, for every step,
// into slot A.slot of A.stages: RK4IP, the stage values y1, k2, k3 and the time-domain fields of
// the four stage inputs; Strang, the time-domain field of the Kerr flow and the state after it.
template <typename T, int LOGN, int R, int C = 1, int METHOD = METHOD_RK4IP>
__global__ void __launch_bounds__(adj_threads<LOGN, R, C>()) segment_kernel(const AdjArgs A)
{
    using GR = Group<T, LOGN, R, C>;
    constexpr int N = GR::N, P = GR::P;
    extern __shared__ __align__(16) unsigned char smem[];
    const StepArgs& a = A.s;
    GR grp;
    bool valid;
    const int inst = adj_setup(grp, smem, a, valid);
    const int t = grp.t;
    const long long off = a.base + (long long)inst * N;
    FieldState<T, LOGN, R, C> fs;
    fs.bind(grp);
    const StepConsts<T> c = step_consts<T>(a, inst, N);
    Props<T, LOGN, R, C> pr;
    pr.init(a, off, t);
    const long long TT = A.total, s = A.seg;
    const long long ns = (A.nsteps - s * A.K < A.K) ? A.nsteps - s * A.K : A.K;
    fs.load(reinterpret_cast<const cx<T>*>(A.ckpt_hi) + A.ckpt_slot * TT + off + t,
            reinterpret_cast<const cx<T>*>(A.ckpt_lo) + A.ckpt_slot * TT + off + t);
    // this thread's slots of step 0 of the segment (surplus groups of a packed block recompute
    // the last instance for the barriers and store nothing); the stage buffer is private to
    // the two roles, so it is indexed by the coalesced scratch slot ts
    cx<T>* out =
        reinterpret_cast<cx<T>*>(A.stages) + A.slot * A.K * ADJ_VECS * TT + off + grp.ts;
    if constexpr (C > 1)
        cluster_sync();   // every block of the cluster runs before the first remote store
    for (long long i = 0; i < ns; ++i) {
        cx<T>* o = out + i * ADJ_VECS * TT;
        if (valid) {
#pragma unroll
            for (int j = 0; j < R; ++j)
                sstore(o + j * P, fs.Dh[j]);
        }
        if constexpr (METHOD == METHOD_RK4IP)
            rk4ip_step_impl<true, rk_cache_ed<T, LOGN, R, C>()>(grp, fs, pr, c,
                                                               valid ? o + TT : nullptr, TT);
        else
            strang_step_impl<true>(grp, fs, pr, c, valid ? o + TT : nullptr, TT);
    }
    // a gradient whose whole trajectory is stored runs its forward pass through this kernel:
    // the segment's final state starts the next segment (or is the final field)
    if (A.out_hi && valid)
        fs.store(reinterpret_cast<cx<T>*>(A.out_hi) + off + t,
                 reinterpret_cast<cx<T>*>(A.out_lo) + off + t);
    if (grp.failed() && a.status)
        a.status[inst] = 2;
    if constexpr (C > 1)
        cluster_sync();   // no block leaves while a peer may still address its shared memory
}

// Backward role: the discrete adjoint of the steps of segment A.seg, last step first, from
// the states, stage values and stage fields in half (A.seg mod 2) of A.stages.  The field cotangent, the
// L cotangents and the pump cotangent are carried between segments in A.dbar, A.gL, A.pbar.
template <typename T, int LOGN, int R, int C = 1>
__global__ void __launch_bounds__(adj_threads<LOGN, R, C>()) adjoint_kernel(const AdjArgs A)
{
    using GR = Group<T, LOGN, R, C>;
    constexpr int N = GR::N, P = GR::P;
    extern __shared__ __align__(16) unsigned char smem[];
    const StepArgs& a = A.s;
    GR grp;
    bool valid;
    const int inst = adj_setup(grp, smem, a, valid);
    const int t = grp.t;
    const long long off = a.base + (long long)inst * N;
    const StepConsts<T> c = step_consts<T>(a, inst, N);
    Props<T, LOGN, R, C> pr;
    pr.init(a, off, t);

    const long long TT = A.total, s = A.seg;
    const long long ns = (A.nsteps - s * A.K < A.K) ? A.nsteps - s * A.K : A.K;
    const cx<T>* buf =
        reinterpret_cast<const cx<T>*>(A.stages) + A.slot * A.K * ADJ_VECS * TT + off + grp.ts;
    cx<T>* dbp = reinterpret_cast<cx<T>*>(A.dbar) + off + t;
    double2* glp = A.gL + off + t;

    cx<T> Db[R];
    LAcc<T> gl[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        Db[j] = dbp[j * P];
        gl[j].init(glp[j * P]);
    }
    // the pump cotangent (thread 0 holds mode 0), accumulated like the L cotangents
    LAcc<T> pb;
    pb.init(t == 0 ? A.pbar[inst] : make_double2(0.0, 0.0));
    const T hh = c.hh, h = c.h, h6 = c.h6, h3 = T(2) * c.h6;
    const T gNn = c.gN;  // g0 / N

    // Prefetch (cluster groups): chunk q = v R + j of step i is the block's PC consecutive
    // slots of vector v, element j, at pf[(buffer i mod 2) CH + q][PC]; thread l reads slot l.
    constexpr bool PF = adj_prefetch<T, LOGN, R, C>();
    constexpr int PC = P / C, CH = ADJ_VECS * R;
    cx<T>* pf = nullptr;
    uint32_t pmb = 0, pph = 0;
    bool pf_failed = false;
    const int l = (int)threadIdx.x;
    if constexpr (PF) {
        pf = reinterpret_cast<cx<T>*>(smem + cluster_smem_bytes<T, LOGN, R, C>());
        pmb = smem_addr(smem + cluster_smem_bytes<T, LOGN, R, C>() +
                        adj_prefetch_bytes<T, LOGN, R, C>());
        if (l == 0) {
            mbar_init(pmb, 1);
            mbar_init(pmb + 8u, 1);
            mbar_init_fence();   // visible to the bulk copies that complete on them
        }
    }
    // copies of step i into buffer i mod 2 (buf - l: the block's first slot)
    auto issue = [&](long long i) {
        const int b = (int)(i & 1);
        if (l == 0)
            mbar_arrive_expect_tx(pmb + 8u * b, (uint32_t)(CH * PC * sizeof(cx<T>)));
        for (int q = l; q < CH; q += PC)
            bulk_g2s(smem_addr(pf + (size_t)(b * CH + q) * PC),
                     buf - l + i * ADJ_VECS * TT + (q / R) * TT + (q % R) * P,
                     (uint32_t)(PC * sizeof(cx<T>)), pmb + 8u * b);
    };
    if constexpr (C > 1)
        cluster_sync();   // every block of the cluster runs before the first remote store
                          // (and this block's threads see its mbarriers initialised)
    if constexpr (PF)
        issue(ns - 1);

    for (long long i = ns - 1; i >= 0; --i) {
        // step i: D, then y1, k2, k3, then a of the stage inputs D, x2, x3, x4, at TT strides
        const cx<T>* Dn = buf + i * ADJ_VECS * TT;
        const cx<T>* sb = nullptr;
        if constexpr (PF) {
            // buffer (i - 1) mod 2 held step i + 1, which every thread has finished with
            __syncthreads();
            if (i >= 1 && !pf_failed) {
                fence_proxy_async_smem();
                issue(i - 1);
            }
            const int b = (int)(i & 1);
            if (!pf_failed && !mbar_wait(pmb + 8u * b, (pph >> b) & 1u, 1 << 20))
                pf_failed = true;   // reported below; the results are then not valid
            pph ^= 1u << b;
            sb = pf + (size_t)b * CH * PC + l;
        }
        // vector v (0: D, 1..3: y1, k2, k3, 4 + st: a of stage input st), element j
        auto ld = [&](int v, int j) -> cx<T> {
            if constexpr (PF)
                return sb[(v * R + j) * PC];
            else
                return Dn[(long long)v * TT + j * P];
        };
        // reverse stages 3 (x4), 2 (x3), 1 (x2), 0 (D)
        cx<T> ub[R], cot[R];
#pragma unroll 1
        for (int st = 3; st >= 0; --st) {
            cx<T> z[R];
            if (st == 3) {
                // cotangent of k4 = F(x4), and the E-cotangent from D' = E w + h/6 k4:
                // conj(hh E) conj(w) Dbar', w = u + h/6 (E y1 + 2 (k2 + k3))
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    const cx<T> E = pr.getE(j);
                    const cx<T> u = cmul(E, ld(0, j));
                    const cx<T> y1 = ld(1, j), k2 = ld(2, j), k3 = ld(3, j);
                    cot[j] = cscale(Db[j], h6);
                    const cx<T> w = caxpy(u, h6, cadd(cmul(E, y1), cscale(cadd(k2, k3), T(2))));
                    gl[j].add(cmulc(cmulc(Db[j], w), cscale(E, hh)));
                }
            }
            if (t == 0) {
                pb.add(cot[0]);
            }
            // zbar = J_F(z)^H cot, a = IDFT(stage input) from the buffer: bbar =
            // IDFT(-i (g0/N) cot), then DFT(2 |a|^2 bbar + a^2 conj(bbar)) (two transforms
            // through one call site)
#pragma unroll
            for (int j = 0; j < R; ++j)
                z[j] = {gNn * cot[j].im, -gNn * cot[j].re};
            grp.out_modes(z);   // the per-mode Kerr factor; F is zero on padding modes,
                                // whose cotangent does not enter
#pragma unroll 1
            for (int p = 0; p < 2; ++p) {
                if (p == 1) {
#pragma unroll
                    for (int j = 0; j < R; ++j) {
                        const cx<T> a = ld(4 + st, j);
                        const cx<T> bb = z[j];                   // bbar
                        const T p2 = a.re * a.re + a.im * a.im;
                        const cx<T> a2 = cmul(a, a);
                        const cx<T> abar = caxpy(cmulc(a2, bb), T(2) * p2, bb);
                        z[j] = cconj(abar);                      // DFT(.) = conj(IDFT(conj .))
                    }
                }
                grp.inverse(z, p);
            }
            grp.mask(z);   // nor does F depend on them: the VJP of m F(m x), m the mask
            // z now holds conj(stage-input cotangent); one loop per stage, so that the stage
            // test is taken once, not per value
            if (st == 0) {
#pragma unroll
                for (int j = 0; j < R; ++j)
                    Db[j] = cadd(Db[j], cconj(z[j]));
            } else if (st == 3) {
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    const cx<T> xb = cconj(z[j]);
                    const cx<T> E = pr.getE(j);
                    const cx<T> wb = cmulc(Db[j], E);            // conj(E) Dbar'
                    const cx<T> hE = cscale(E, hh);
                    const cx<T> u = cmul(E, ld(0, j));
                    const cx<T> v = caxpy(u, h, ld(3, j));
                    const cx<T> vb = cmulc(xb, E);               // conj(E) x4bar
                    gl[j].add(cmulc(cmulc(xb, v), hE));          // conj(hh E) conj(v) x4bar
                    ub[j] = cadd(wb, vb);
                    cot[j] = caxpy(cscale(wb, h3), h, vb);       // k3bar
                }
            } else if (st == 2) {
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    const cx<T> xb = cconj(z[j]);
                    const cx<T> wb = cmulc(Db[j], pr.getE(j));   // conj(E) Dbar'
                    ub[j] = cadd(ub[j], xb);
                    cot[j] = caxpy(cscale(wb, h3), hh, xb);      // k2bar
                }
            } else {   // st == 1
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    const cx<T> xb = cconj(z[j]);
                    const cx<T> E = pr.getE(j);
                    const cx<T> wb = cmulc(Db[j], E);            // conj(E) Dbar'
                    const cx<T> hE = cscale(E, hh);
                    ub[j] = cadd(ub[j], xb);
                    const cx<T> k1b = caxpy(cscale(wb, h6), hh, xb);
                    const cx<T> y1 = ld(1, j);
                    const cx<T> D = ld(0, j);
                    // conj(hh E) (conj(D) ubar + conj(y1) k1bar): one term, one sum
                    gl[j].add(cmulc(cadd(cmulc(ub[j], D), cmulc(k1b, y1)), hE));
                    Db[j] = cmulc(ub[j], E);                     // conj(E) ubar
                    cot[j] = cmulc(k1b, E);                      // y1bar = conj(E) k1bar
                }
            }
        }
    }
    if (valid) {
#pragma unroll
        for (int j = 0; j < R; ++j) {
            dbp[j * P] = Db[j];
            glp[j * P] = gl[j].finish(glp[j * P]);
        }
        if (t == 0)
            A.pbar[inst] = pb.finish(A.pbar[inst]);
    }
    if ((grp.failed() || pf_failed) && a.status)
        a.status[inst] = 2;
    if constexpr (C > 1)
        cluster_sync();   // no block leaves while a peer may still address its shared memory
}

// Backward role of the Strang split step (Sec. 2, split-step Fourier method with the field in
// the frequency domain): the discrete adjoint of the steps of segment A.seg, last step first,
// from the states D, the time-domain fields a of the Kerr flow and the states D2 after it in
// half (A.seg mod 2) of A.stages.  One step of the forward kernels is
//     D1 = E D + c,  a = IDFT(D1),  D2 = D1 + m DFT(a (u - 1)) / N,  D3 = E D2 + c,
// with E = exp(L h/2), c the pump increment of the linear half flow on mu = 0,
// u = exp(i g0 h |a|^2) and m the physical modes.  In reverse:
//     D2bar = conj(E) D3bar,            Lbar += conj(h/2 E) conj(D2) D3bar,  cbar += D3bar_0;
//     bbar = IDFT(m D2bar) / N,
//     abar = (conj(u) (1 - i g0 h |a|^2) - 1) bbar + i g0 h a^2 u conj(bbar),
//     D1bar = D2bar + m DFT(abar),
//     Dbar = conj(E) D1bar,             Lbar += conj(h/2 E) conj(D) D1bar,   cbar += D1bar_0.
// cbar accumulates in A.pbar; the host turns it into the cotangents of the pump and of L_0 (the
// increment c depends on both) once all segments are done.  Two transforms per step.
template <typename T, int LOGN, int R, int C = 1>
__global__ void __launch_bounds__(adj_threads<LOGN, R, C>()) strang_adjoint_kernel(const AdjArgs A)
{
    using GR = Group<T, LOGN, R, C>;
    constexpr int N = GR::N, P = GR::P;
    extern __shared__ __align__(16) unsigned char smem[];
    const StepArgs& a = A.s;
    GR grp;
    bool valid;
    const int inst = adj_setup(grp, smem, a, valid);
    const int t = grp.t;
    const long long off = a.base + (long long)inst * N;
    const StepConsts<T> c = step_consts<T>(a, inst, N);
    Props<T, LOGN, R, C> pr;
    pr.init(a, off, t);

    const long long TT = A.total, s = A.seg;
    const long long ns = (A.nsteps - s * A.K < A.K) ? A.nsteps - s * A.K : A.K;
    const cx<T>* buf =
        reinterpret_cast<const cx<T>*>(A.stages) + A.slot * A.K * ADJ_VECS * TT + off + grp.ts;
    cx<T>* dbp = reinterpret_cast<cx<T>*>(A.dbar) + off + t;
    double2* glp = A.gL + off + t;

    cx<T> Db[R];
    LAcc<T> gl[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        Db[j] = dbp[j * P];
        gl[j].init(glp[j * P]);
    }
    // the pump cotangent (thread 0 holds mode 0), accumulated like the L cotangents
    LAcc<T> pb;
    pb.init(t == 0 ? A.pbar[inst] : make_double2(0.0, 0.0));
    const T hh = c.hh;
    const T gh = T(2) * c.g0h;                // g0 h
    constexpr T invN = (T)(1.0 / (1 << LOGN));
    if constexpr (C > 1)
        cluster_sync();   // every block of the cluster runs before the first remote store

    for (long long i = ns - 1; i >= 0; --i) {
        // step i: D, a, D2 at TT strides
        const cx<T>* Dn = buf + i * ADJ_VECS * TT;
        // second linear half flow
        if (t == 0) {
            pb.add(Db[0]);
        }
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const cx<T> E = pr.getE(j);
            gl[j].add(cmulc(cmulc(Db[j], Dn[2 * TT + j * P]), cscale(E, hh)));
            Db[j] = cmulc(Db[j], E);                                 // D2bar
        }
        // Kerr flow
        cx<T> z[R];
#pragma unroll
        for (int j = 0; j < R; ++j)
            z[j] = Db[j];
        grp.mask(z);
#pragma unroll 1
        for (int p = 0; p < 2; ++p) {
            if (p == 1) {
                // sin and cos of half the phase, as the forward step takes them (the Taylor
                // series for every value, sincosf behind one branch per thread)
                cx<T> avs[R];
                T p2s[R], sns[R], css[R];
                bool big = false;
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    avs[j] = Dn[TT + j * P];
                    p2s[j] = avs[j].re * avs[j].re + avs[j].im * avs[j].im;
                    if constexpr (sizeof(T) == 4) {
                        taylor_sincos(c.g0h * p2s[j], sns[j], css[j]);
                        big |= !small_phase(c.g0h * p2s[j]);
                    } else {
                        sincos(c.g0h * p2s[j], &sns[j], &css[j]);
                    }
                }
                if constexpr (sizeof(T) == 4) {
                    if (big) {
#pragma unroll
                        for (int j = 0; j < R; ++j)
                            if (!small_phase(c.g0h * p2s[j]))
                                sincosf(c.g0h * p2s[j], &sns[j], &css[j]);
                    }
                }
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    const cx<T> av = avs[j];
                    const T p2 = p2s[j];
                    const T sn = sns[j], cs = css[j];
                    const T ph = gh * p2;                            // g0 h |a|^2
                    const T ur = T(1) - T(2) * sn * sn, ui = T(2) * sn * cs;
                    const cx<T> bb = cscale(z[j], invN);             // bbar
                    // conj(u) (1 - i ph) - 1
                    const cx<T> A1 = {T(-2) * sn * sn - ui * ph, -ph * ur - ui};
                    // i g0 h a^2 u
                    const cx<T> au = cmul(cmul(av, av), cx<T>{ur, ui});
                    const cx<T> B1 = {-gh * au.im, gh * au.re};
                    const cx<T> ab = cadd(cmul(A1, bb), cmulc(B1, bb));
                    z[j] = cconj(ab);                                // DFT(.) = conj(IDFT(conj .))
                }
            }
            grp.inverse(z, p);
        }
        grp.mask(z);
#pragma unroll
        for (int j = 0; j < R; ++j)
            Db[j] = cadd(Db[j], cconj(z[j]));                        // D1bar
        // first linear half flow
        if (t == 0) {
            pb.add(Db[0]);
        }
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const cx<T> E = pr.getE(j);
            gl[j].add(cmulc(cmulc(Db[j], Dn[j * P]), cscale(E, hh)));
            Db[j] = cmulc(Db[j], E);                                 // Dbar
        }
    }
    if (valid) {
#pragma unroll
        for (int j = 0; j < R; ++j) {
            dbp[j * P] = Db[j];
            glp[j * P] = gl[j].finish(glp[j * P]);
        }
        if (t == 0)
            A.pbar[inst] = pb.finish(A.pbar[inst]);
    }
    if (grp.failed() && a.status)
        a.status[inst] = 2;
    if constexpr (C > 1)
        cluster_sync();   // no block leaves while a peer may still address its shared memory
}

}  // namespace cme
