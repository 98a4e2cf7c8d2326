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
// Memory: the forward pass stores the field at the start of every segment of K steps
// (checkpoints); the backward kernel recomputes one segment at a time from its checkpoint
// into a segment buffer, then walks it backwards.
#pragma once

#include "cme_adjoint_args.h"
#include "cme_step.cuh"

namespace cme {

template <typename T>
CME_DEV cx<T> cconj(cx<T> a) { return {a.re, -a.im}; }

template <typename T, int LOGN, int R>
__global__ void __launch_bounds__(max_threads<LOGN, R>()) adjoint_kernel(const AdjArgs A)
{
    using GR = Group<T, LOGN, R>;
    constexpr int N = GR::N, P = GR::P;
    extern __shared__ __align__(16) unsigned char smem[];
    const StepArgs& a = A.s;

    const int g = threadIdx.x / P;
    int inst = blockIdx.x * a.G + g;
    const bool valid = inst < a.ninst;
    if (!valid)
        inst = a.ninst - 1;
    GR grp;
    grp.setup(smem, g, threadIdx.x - g * P, a.tw);
    const int t = grp.t;
    const long long off = a.base + (long long)inst * N;

    FieldState<T, LOGN, R> fs;
    fs.bind(grp);
    const StepConsts<T> c = step_consts<T>(a, inst, N);
    Props<T, LOGN, R> pr;
    pr.init(a, off, t);

    cx<T>* seg = reinterpret_cast<cx<T>*>(A.seg) + off + t;
    cx<T>* yb = reinterpret_cast<cx<T>*>(A.ybuf) + off + t;
    cx<T>* dbp = reinterpret_cast<cx<T>*>(A.dbar) + off + t;
    const long long TT = A.total;

    cx<T> Db[R];
    double2 gl[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        Db[j] = dbp[j * P];
        gl[j] = make_double2(0.0, 0.0);
    }
    double2 pb = make_double2(0.0, 0.0);
    const T hh = c.hh, h = c.h, h6 = c.h6, h3 = T(2) * c.h6;
    const T gNn = c.gN;  // g0 / N

    for (long long s = A.S - 1; s >= 0; --s) {
        const long long n0 = s * A.K;
        const long long ns = (A.nsteps - n0 < A.K) ? A.nsteps - n0 : A.K;
        // recompute the segment's states from its checkpoint
        fs.load(reinterpret_cast<const cx<T>*>(A.ckpt_hi) + s * TT + off + t,
                reinterpret_cast<const cx<T>*>(A.ckpt_lo) + s * TT + off + t);
        for (long long i = 0; i < ns; ++i) {
#pragma unroll
            for (int j = 0; j < R; ++j)
                seg[i * TT + j * P] = fs.Dh[j];
            if (i + 1 < ns)
                rk4ip_step(grp, fs, pr, c);
        }
        // walk the segment backwards
        for (long long i = ns - 1; i >= 0; --i) {
            const cx<T>* Dn = seg + i * TT;
            // forward stage values of step i: y1 = F(D), k2 = F(x2), k3 = F(x3)
            cx<T> x[R];
#pragma unroll
            for (int j = 0; j < R; ++j)
                x[j] = Dn[j * P];
#pragma unroll 1
            for (int st = 0; st < 3; ++st) {
                grp.rhs(x, c.gN, c.pump);
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    yb[st * TT + j * P] = x[j];
                    const cx<T> E = pr.getE(j);
                    const cx<T> u = cmul(E, Dn[j * P]);
                    if (st == 0)
                        x[j] = caxpy(u, hh, cmul(E, x[j]));        // x2 = u + h/2 E y1
                    else if (st == 1)
                        x[j] = caxpy(u, hh, x[j]);                  // x3 = u + h/2 k2
                }
            }
            // reverse stages 3 (x4), 2 (x3), 1 (x2), 0 (D)
            cx<T> ub[R], cot[R];
#pragma unroll 1
            for (int st = 3; st >= 0; --st) {
                cx<T> z[R];
                // stage input and the cotangent of its F output
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    const cx<T> E = pr.getE(j);
                    const cx<T> D = Dn[j * P];
                    const cx<T> u = cmul(E, D);
                    if (st == 3) {
                        const cx<T> y1 = yb[j * P], k2 = yb[TT + j * P], k3 = yb[2 * TT + j * P];
                        const cx<T> v = caxpy(u, h, k3);
                        z[j] = cmul(E, v);                           // x4 = E (u + h k3)
                        cot[j] = cscale(Db[j], h6);                  // k4bar
                        // E-cotangent from D' = E w + ...: conj(w) Dbar'
                        const cx<T> w = caxpy(u, h6, cadd(cmul(E, y1), cscale(cadd(k2, k3), T(2))));
                        const cx<T> lb = cmulc(cmulc(Db[j], w), cscale(E, hh));   // conj(hh E) conj(w) Db
                        gl[j].x += (double)lb.re;
                        gl[j].y += (double)lb.im;
                    } else if (st == 2) {
                        z[j] = caxpy(u, hh, yb[TT + j * P]);         // x3
                    } else if (st == 1) {
                        z[j] = caxpy(u, hh, cmul(E, yb[j * P]));     // x2
                    } else {
                        z[j] = D;
                    }
                }
                if (t == 0) {
                    pb.x += (double)cot[0].re;
                    pb.y += (double)cot[0].im;
                }
                // zbar = J_F(z)^H cot  (three transforms through one call site)
                cx<T> aa[R];
#pragma unroll 1
                for (int p = 0; p < 3; ++p) {
                    if (p == 1) {
#pragma unroll
                        for (int j = 0; j < R; ++j) {
                            aa[j] = z[j];                            // a = IDFT(stage input)
                            // -i (g0/N) cot
                            z[j] = {gNn * cot[j].im, -gNn * cot[j].re};
                        }
                    } else if (p == 2) {
#pragma unroll
                        for (int j = 0; j < R; ++j) {
                            const cx<T> bb = z[j];                   // bbar
                            const T p2 = aa[j].re * aa[j].re + aa[j].im * aa[j].im;
                            const cx<T> a2 = cmul(aa[j], aa[j]);
                            const cx<T> ab = caxpy(cmulc(a2, bb), T(2) * p2, bb);
                            z[j] = cconj(ab);                        // DFT(ab) = conj(IDFT(conj ab))
                        }
                    }
                    grp.inverse(z);
                }
                // z now holds conj(stage-input cotangent)
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    const cx<T> xb = cconj(z[j]);
                    const cx<T> E = pr.getE(j);
                    const cx<T> D = Dn[j * P];
                    const cx<T> u = cmul(E, D);
                    const cx<T> wb = cmulc(Db[j], E);                // conj(E) Dbar'
                    const cx<T> hE = cscale(E, hh);
                    if (st == 3) {
                        const cx<T> v = caxpy(u, h, yb[2 * TT + j * P]);
                        const cx<T> vb = cmulc(xb, E);               // conj(E) x4bar
                        const cx<T> lb = cmulc(cmulc(xb, v), hE);    // conj(hh E) conj(v) x4bar
                        gl[j].x += (double)lb.re;
                        gl[j].y += (double)lb.im;
                        ub[j] = cadd(wb, vb);
                        cot[j] = caxpy(cscale(wb, h3), h, vb);       // k3bar
                    } else if (st == 2) {
                        ub[j] = cadd(ub[j], xb);
                        cot[j] = caxpy(cscale(wb, h3), hh, xb);      // k2bar
                    } else if (st == 1) {
                        ub[j] = cadd(ub[j], xb);
                        const cx<T> k1b = caxpy(cscale(wb, h6), hh, xb);
                        const cx<T> y1 = yb[j * P];
                        const cx<T> l1 = cmulc(cmulc(ub[j], D), hE);  // conj(hh E) conj(D) ubar
                        const cx<T> l2 = cmulc(cmulc(k1b, y1), hE);   // conj(hh E) conj(y1) k1bar
                        gl[j].x += (double)l1.re + (double)l2.re;
                        gl[j].y += (double)l1.im + (double)l2.im;
                        Db[j] = cmulc(ub[j], E);                     // conj(E) ubar
                        cot[j] = cmulc(k1b, E);                      // y1bar = conj(E) k1bar
                    } else {
                        Db[j] = cadd(Db[j], xb);
                    }
                }
            }
        }
    }
    if (valid) {
        double2* glp = A.gL + off + t;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            dbp[j * P] = Db[j];
            glp[j * P] = gl[j];
        }
        if (t == 0)
            A.pbar[inst] = pb;
    }
}

}  // namespace cme
