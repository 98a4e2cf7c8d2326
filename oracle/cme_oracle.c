/*
 * FP64 CPU oracle for the coupled mode equations (CMEs) of Kerr comb generation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may load this library.  It shares no code with the CUDA path.
 *
 * Everything here is the plain definition, written for reading, not for speed:
 *   - the four-wave-mixing (FWM) sum is the direct triple sum of Eq. 2 / Eq. 3,
 *     O(N^3) per evaluation (the cost analysed in Sec. 2 of the paper);
 *   - transforms, where the Strang splitting needs the time-domain field, are the naive
 *     O(N^2) sums over the mode number mu of Eq. 4;
 *   - RK4IP (fourth-order Runge-Kutta in the interaction picture), the Strang split step
 *     and plain RK4 take their steps in the textbook order.
 *
 * Layout: every complex array holds modes in centred order, index i <-> mu = i - N/2.
 *
 * Model (Eq. 1 written in the frame D_mu = A_mu exp(i (omega_mu - omega_0 - sigma) tau),
 * which removes every explicit time dependence of Eq. 1 because alpha - beta + gamma = mu):
 *     dD_mu/dtau = L_mu D_mu + F_mu(D),
 *     L_mu = -kappa_mu/2 + i (omega_mu - omega_0 - sigma),
 *     F_mu(D) = delta_{mu,0} sqrt(kappa_ext) A_in + i g0 FWM_mu(D),
 *     (optionally a per-mode g0_mu in place of g0: a frequency-dependent Kerr coefficient of
 *     the output mode, Sec. 2 noting that a constant g0 is no necessary restriction),
 *     FWM_mu(D) = sum_{alpha - beta + gamma = mu} D_alpha conj(D_beta) D_gamma.
 * The constraint alpha - beta + gamma = mu is taken modulo N ("circular", the reading that
 * matches Eq. 4 with an N-point transform) or literally ("linear", no wrap-around).
 *
 * Physical modes (the zero padding of Sec. 2: 201 modes in a 256-point transform): of the N
 * modes only the M centred ones, mu = -floor(M/2) .. M - floor(M/2) - 1, are physical.  The
 * others are held at zero: the FWM sum runs over physical alpha, beta, gamma only and is
 * evaluated on physical mu only, and the Strang Kerr step is followed by zeroing them.
 * M = N is the unpadded system.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define ORACLE_OK 0
#define ORACLE_EINVAL -1

/* centred index of mode mu, wrapped modulo N */
static int wrap_index(long mu, int N)
{
    long i = (mu + N / 2) % N;
    if (i < 0)
        i += N;
    return (int)i;
}

static void load(int N, const double* in, cplx* out)
{
    for (int i = 0; i < N; ++i)
        out[i] = in[2 * i] + I * in[2 * i + 1];
}

static void store(int N, const cplx* in, double* out)
{
    for (int i = 0; i < N; ++i) {
        out[2 * i] = creal(in[i]);
        out[2 * i + 1] = cimag(in[i]);
    }
}

/* Is centred index i (mu = i - N/2) one of the M physical modes? */
static int physical(int i, int N, int M)
{
    const int first = N / 2 - M / 2;
    return i >= first && i < first + M;
}

/* Eq. 2 / Eq. 3: direct sum over (beta, gamma) with alpha = mu + beta - gamma, over the M
 * physical modes. */
static void fwm_direct(int N, int linear, int M, const cplx* D, cplx* out)
{
    const int h = N / 2;
    for (int mu = -h; mu < N - h; ++mu) {
        cplx s = 0.0;
        if (!physical(mu + h, N, M)) {
            out[mu + h] = 0.0;
            continue;
        }
        for (int beta = -h; beta < N - h; ++beta) {
            if (!physical(beta + h, N, M))
                continue;
            const cplx cb = conj(D[beta + h]);
            for (int gamma = -h; gamma < N - h; ++gamma) {
                if (!physical(gamma + h, N, M))
                    continue;
                long alpha = (long)mu + beta - gamma;
                int ia;
                if (linear) {
                    if (alpha < -h || alpha >= N - h)
                        continue;
                    ia = (int)(alpha + h);
                } else {
                    ia = wrap_index(alpha, N);
                }
                if (!physical(ia, N, M))
                    continue;
                s += D[ia] * cb * D[gamma + h];
            }
        }
        out[mu + h] = s;
    }
}

typedef struct {
    int N;
    int linear;
    int M;   /* physical modes (N: all) */
    const double* kappa;
    const double* omega;
    double g0;
    double kappa_ext;
    cplx A_in;
    double sigma;
    const double* g0mu;   /* per-mode Kerr coefficients g0_mu (centred), or NULL: g0 on every mode */
} model;

/* Kerr coefficient of the four-wave-mixing term of output mode i (centred index). */
static double kerr_coef(const model* m, int i)
{
    return m->g0mu ? m->g0mu[i] : m->g0;
}

/* F(D) = pump + i g0 FWM(D); with per-mode coefficients F_mu = pump + i g0_mu FWM_mu(D) */
static void rhs_nonlinear(const model* m, const cplx* D, cplx* out)
{
    fwm_direct(m->N, m->linear, m->M, D, out);
    for (int i = 0; i < m->N; ++i)
        out[i] *= I * kerr_coef(m, i);
    out[m->N / 2] += sqrt(m->kappa_ext) * m->A_in;
}

static cplx lin_coef(const model* m, int i)
{
    const double omega0 = m->omega[m->N / 2];
    return -0.5 * m->kappa[i] + I * (m->omega[i] - omega0 - m->sigma);
}

/* One RK4IP step (Hult, J. Lightwave Technol. 25, 3770 (2007)) with E = exp(L h/2). */
static void step_rk4ip(const model* m, double h, cplx* D, cplx* w)
{
    const int N = m->N;
    cplx *E = w, *AI = w + N, *k1 = w + 2 * N, *k2 = w + 3 * N, *k3 = w + 4 * N,
         *k4 = w + 5 * N, *x = w + 6 * N;
    for (int i = 0; i < N; ++i)
        E[i] = cexp(lin_coef(m, i) * (0.5 * h));
    for (int i = 0; i < N; ++i)
        AI[i] = E[i] * D[i];
    rhs_nonlinear(m, D, k1);
    for (int i = 0; i < N; ++i)
        k1[i] *= E[i];
    for (int i = 0; i < N; ++i)
        x[i] = AI[i] + 0.5 * h * k1[i];
    rhs_nonlinear(m, x, k2);
    for (int i = 0; i < N; ++i)
        x[i] = AI[i] + 0.5 * h * k2[i];
    rhs_nonlinear(m, x, k3);
    for (int i = 0; i < N; ++i)
        x[i] = E[i] * (AI[i] + h * k3[i]);
    rhs_nonlinear(m, x, k4);
    for (int i = 0; i < N; ++i)
        D[i] = E[i] * (AI[i] + h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i])) + h / 6.0 * k4[i];
}

/* Classic RK4 on the full right-hand side L D + F(D). */
static void full_rhs(const model* m, const cplx* D, cplx* out)
{
    rhs_nonlinear(m, D, out);
    for (int i = 0; i < m->N; ++i)
        out[i] += lin_coef(m, i) * D[i];
}

static void step_rk4(const model* m, double h, cplx* D, cplx* w)
{
    const int N = m->N;
    cplx *k1 = w, *k2 = w + N, *k3 = w + 2 * N, *k4 = w + 3 * N, *x = w + 4 * N;
    full_rhs(m, D, k1);
    for (int i = 0; i < N; ++i)
        x[i] = D[i] + 0.5 * h * k1[i];
    full_rhs(m, x, k2);
    for (int i = 0; i < N; ++i)
        x[i] = D[i] + 0.5 * h * k2[i];
    full_rhs(m, x, k3);
    for (int i = 0; i < N; ++i)
        x[i] = D[i] + h * k3[i];
    full_rhs(m, x, k4);
    for (int i = 0; i < N; ++i)
        D[i] += h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

/* Naive transform over the mode number (Eq. 4 without the FFT):
 *   sign=+1: a_j = sum_mu D_mu exp(+2 pi i j mu / N)          (time samples, j = 0..N-1)
 *   sign=-1: D_mu = sum_j a_j exp(-2 pi i j mu / N)           (mode amplitudes, centred)
 * The "time" array is indexed by j = 0..N-1. */
static void dft_modes_to_time(int N, const cplx* D, cplx* a)
{
    for (int j = 0; j < N; ++j) {
        cplx s = 0.0;
        for (int i = 0; i < N; ++i) {
            const long mu = i - N / 2;
            const long e = ((long)j * mu) % N;
            s += D[i] * cexp(I * (2.0 * M_PI * (double)e / (double)N));
        }
        a[j] = s;
    }
}

static void dft_time_to_modes(int N, const cplx* a, cplx* D)
{
    for (int i = 0; i < N; ++i) {
        const long mu = i - N / 2;
        cplx s = 0.0;
        for (int j = 0; j < N; ++j) {
            const long e = ((long)j * mu) % N;
            s += a[j] * cexp(-I * (2.0 * M_PI * (double)e / (double)N));
        }
        D[i] = s;
    }
}

/* Exact solution of the linear part dD/dtau = L D + delta_{mu,0} p over a time dt. */
static void linear_substep(const model* m, double dt, cplx* D)
{
    const int N = m->N;
    const cplx p = sqrt(m->kappa_ext) * m->A_in;
    for (int i = 0; i < N; ++i) {
        const cplx L = lin_coef(m, i);
        const cplx e = cexp(L * dt);
        D[i] = e * D[i];
        if (i == N / 2) {
            if (cabs(L) == 0.0)
                D[i] += dt * p;
            else
                D[i] += (e - 1.0) / L * p;
        }
    }
}

/* Strang split step: linear half step, exact Kerr step in the time domain, linear half step.
 * With a = (unnormalised) inverse transform of D, the nonlinear flow of the circular CME is
 * da_j/dtau = i g0 |a_j|^2 a_j, whose exact solution keeps |a_j| and rotates the phase. */
static void step_strang(const model* m, double h, cplx* D, cplx* w)
{
    const int N = m->N;
    cplx* a = w;
    linear_substep(m, 0.5 * h, D);
    dft_modes_to_time(N, D, a);
    for (int j = 0; j < N; ++j) {
        const double p2 = creal(a[j]) * creal(a[j]) + cimag(a[j]) * cimag(a[j]);
        a[j] *= cexp(I * (m->g0 * p2 * h));
    }
    dft_time_to_modes(N, a, D);
    for (int i = 0; i < N; ++i)
        D[i] = physical(i, N, m->M) ? D[i] / (double)N : 0.0;
    linear_substep(m, 0.5 * h, D);
}

static int check_model(int N, const double* kappa, const double* omega)
{
    if (N < 1 || !kappa || !omega)
        return ORACLE_EINVAL;
    return ORACLE_OK;
}

/* ---------------------------------------------------------------------------------------
 * Exported entry points (plain doubles; complex arrays interleaved re, im).
 * ------------------------------------------------------------------------------------- */

int oracle_fwm(int N, int linear, int M, const double* D, double* out)
{
    if (N < 1 || M < 1 || M > N || !D || !out)
        return ORACLE_EINVAL;
    cplx* d = malloc(sizeof(cplx) * 2 * N);
    load(N, D, d);
    fwm_direct(N, linear, M, d, d + N);
    store(N, d + N, out);
    free(d);
    return ORACLE_OK;
}

/* F(D) = delta_{mu,0} sqrt(kappa_ext) A_in + i g0 FWM(D) (g0mu: per-mode g0_mu, or NULL) */
int oracle_rhs(int N, int linear, int M, double g0, const double* g0mu, double kappa_ext,
               double ain_re, double ain_im, const double* D, double* out)
{
    if (N < 1 || M < 1 || M > N || !D || !out)
        return ORACLE_EINVAL;
    model m = {N, linear, M, NULL, NULL, g0, kappa_ext, ain_re + I * ain_im, 0.0, g0mu};
    cplx* d = malloc(sizeof(cplx) * 2 * N);
    load(N, D, d);
    rhs_nonlinear(&m, d, d + N);
    store(N, d + N, out);
    free(d);
    return ORACLE_OK;
}

/* method: 0 = RK4IP, 1 = Strang, 2 = plain RK4.  D (2N doubles) is advanced in place.
 * g0mu: per-mode Kerr coefficients (N, centred) or NULL; the Strang step has no exact Kerr flow
 * with per-mode coefficients and refuses them. */
int oracle_integrate(int method, int N, int linear, int M, const double* kappa,
                     const double* omega, double g0, const double* g0mu, double kappa_ext,
                     double ain_re, double ain_im, double sigma, double h, long nsteps,
                     double* D)
{
    if (check_model(N, kappa, omega) || !D || nsteps < 0 || method < 0 || method > 2 || M < 1 ||
        M > N)
        return ORACLE_EINVAL;
    if (method == 1 && (linear || g0mu))
        return ORACLE_EINVAL;
    model m = {N, linear, M, kappa, omega, g0, kappa_ext, ain_re + I * ain_im, sigma, g0mu};
    cplx* d = malloc(sizeof(cplx) * N);
    cplx* w = malloc(sizeof(cplx) * 8 * N);
    load(N, D, d);
    for (int i = 0; i < N; ++i)   /* padding modes start (and stay) at zero */
        if (!physical(i, N, M))
            d[i] = 0.0;
    for (long n = 0; n < nsteps; ++n) {
        if (method == 0)
            step_rk4ip(&m, h, d, w);
        else if (method == 1)
            step_strang(&m, h, d, w);
        else
            step_rk4(&m, h, d, w);
    }
    store(N, d, D);
    free(d);
    free(w);
    return ORACLE_OK;
}

/* Eq. 1 exactly as printed, in the laboratory frame with its explicit phase factors:
 *   dA_mu/dtau = -kappa_mu/2 A_mu + delta_{mu,0} sqrt(kappa_ext) A_in exp(i sigma tau)
 *              + i g0 sum_{alpha-beta+gamma=mu} A_alpha conj(A_beta) A_gamma
 *                      exp(i (omega_alpha - omega_beta + omega_gamma - omega_mu) tau),
 * integrated with classic RK4 from tau0.  Used to pin the change of frame. */
static void rhs_eq1(const model* m, double tau, const cplx* A, cplx* out)
{
    const int N = m->N, hN = N / 2;
    for (int mu = -hN; mu < N - hN; ++mu) {
        cplx s = 0.0;
        for (int beta = -hN; beta < N - hN; ++beta) {
            for (int gamma = -hN; gamma < N - hN; ++gamma) {
                long alpha = (long)mu + beta - gamma;
                int ia;
                if (m->linear) {
                    if (alpha < -hN || alpha >= N - hN)
                        continue;
                    ia = (int)(alpha + hN);
                } else {
                    ia = wrap_index(alpha, N);
                }
                const double ph = m->omega[ia] - m->omega[beta + hN] + m->omega[gamma + hN]
                                  - m->omega[mu + hN];
                s += A[ia] * conj(A[beta + hN]) * A[gamma + hN] * cexp(I * ph * tau);
            }
        }
        out[mu + hN] = -0.5 * m->kappa[mu + hN] * A[mu + hN] + I * m->g0 * s;
    }
    out[hN] += sqrt(m->kappa_ext) * m->A_in * cexp(I * m->sigma * tau);
}

int oracle_integrate_eq1(int N, int linear, const double* kappa, const double* omega, double g0,
                         double kappa_ext, double ain_re, double ain_im, double sigma,
                         double tau0, double h, long nsteps, double* A)
{
    if (check_model(N, kappa, omega) || !A || nsteps < 0)
        return ORACLE_EINVAL;
    model m = {N, linear, N, kappa, omega, g0, kappa_ext, ain_re + I * ain_im, sigma};
    cplx* a = malloc(sizeof(cplx) * 6 * N);
    cplx *k1 = a + N, *k2 = a + 2 * N, *k3 = a + 3 * N, *k4 = a + 4 * N, *x = a + 5 * N;
    load(N, A, a);
    double tau = tau0;
    for (long n = 0; n < nsteps; ++n) {
        rhs_eq1(&m, tau, a, k1);
        for (int i = 0; i < N; ++i)
            x[i] = a[i] + 0.5 * h * k1[i];
        rhs_eq1(&m, tau + 0.5 * h, x, k2);
        for (int i = 0; i < N; ++i)
            x[i] = a[i] + 0.5 * h * k2[i];
        rhs_eq1(&m, tau + 0.5 * h, x, k3);
        for (int i = 0; i < N; ++i)
            x[i] = a[i] + h * k3[i];
        rhs_eq1(&m, tau + h, x, k4);
        for (int i = 0; i < N; ++i)
            a[i] += h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
        tau = tau0 + (double)(n + 1) * h;
    }
    store(N, a, A);
    free(a);
    return ORACLE_OK;
}

/* Naive transform over the mode number.  sign=+1: modes -> time; sign=-1: time -> modes. */
int oracle_dft(int N, int sign, const double* in, double* out)
{
    if (N < 1 || !in || !out || (sign != 1 && sign != -1))
        return ORACLE_EINVAL;
    cplx* d = malloc(sizeof(cplx) * 2 * N);
    load(N, in, d);
    if (sign == 1)
        dft_modes_to_time(N, d, d + N);
    else
        dft_time_to_modes(N, d, d + N);
    store(N, d + N, out);
    free(d);
    return ORACLE_OK;
}

/* Conserved quantities of the lossless, unpumped system (kappa = 0, A_in = 0):
 *   out[0] = sum_mu |D_mu|^2
 *   out[1] = H = sum_mu (omega_mu - omega_0 - sigma) |D_mu|^2 + (g0/2) sum_mu conj(D_mu) FWM_mu(D)
 * with dD_mu/dtau = i dH/d conj(D_mu). */
int oracle_invariants(int N, int linear, const double* omega, double g0, double sigma,
                      const double* D, double* out)
{
    if (N < 1 || !omega || !D || !out)
        return ORACLE_EINVAL;
    cplx* d = malloc(sizeof(cplx) * 2 * N);
    load(N, D, d);
    fwm_direct(N, linear, N, d, d + N);
    double norm = 0.0, quad = 0.0;
    cplx quart = 0.0;
    for (int i = 0; i < N; ++i) {
        const double p = creal(d[i]) * creal(d[i]) + cimag(d[i]) * cimag(d[i]);
        norm += p;
        quad += (omega[i] - omega[N / 2] - sigma) * p;
        quart += conj(d[i]) * d[N + i];
    }
    out[0] = norm;
    out[1] = quad + 0.5 * g0 * creal(quart);
    free(d);
    return ORACLE_OK;
}

/* ---------------------------------------------------------------------------------------
 * Discrete adjoint of the RK4IP map (reverse mode through exactly the steps of step_rk4ip),
 * for the log-power-spectrum misfit loss
 *     L = sum_mu (log10(|D_mu|^2 + eps) - T_mu)^2     at the final step.
 * Cotangents of complex quantities follow vbar = dL/dRe v + i dL/dIm v, so that for y = a x
 * (complex product) xbar += conj(a) ybar and abar += conj(x) ybar.
 *
 * VJP of the FWM sum, from its definition FWM_mu = sum_{beta,gamma} D_{mu+beta-gamma}
 * conj(D_beta) D_gamma (indices modulo N or linear):
 *     Dbar_nu = 2 sum_{mu,beta} Wbar_mu D_beta conj(D_{mu+beta-nu})
 *             +   sum_{mu,gamma} conj(Wbar_mu) D_{mu+nu-gamma} D_gamma .
 * Outputs: gD0 (cotangent of the initial field), gLi / gLr (dL/dIm L_mu and dL/dRe L_mu summed
 * over all steps, L_mu = -kappa_mu/2 + i(omega_mu - omega_0 - sigma)) and gP (cotangent of the
 * pump sqrt(kappa_ext) A_in).
 * ------------------------------------------------------------------------------------- */
/* centred index of alpha (wrapped or linear), or -1 if it is not a physical mode */
static int idx_of(long alpha, int N, int linear, int M)
{
    const int h = N / 2;
    int i;
    if (linear) {
        if (alpha < -h || alpha >= N - h)
            return -1;
        i = (int)(alpha + h);
    } else {
        i = wrap_index(alpha, N);
    }
    return physical(i, N, M) ? i : -1;
}

/* Over physical modes only: mu, nu, beta, gamma and the derived index all physical (the FWM
 * sum of the padded system does not depend on the padding modes, nor does it feed them). */
static void fwm_vjp(int N, int linear, int M, const cplx* D, const cplx* Wbar, cplx* Dbar)
{
    const int h = N / 2;
    for (int nu = -h; nu < N - h; ++nu) {
        cplx s = 0.0;
        if (!physical(nu + h, N, M)) {
            Dbar[nu + h] = 0.0;
            continue;
        }
        for (int mu = -h; mu < N - h; ++mu) {
            if (!physical(mu + h, N, M))
                continue;
            const cplx w = Wbar[mu + h];
            for (int beta = -h; beta < N - h; ++beta) {
                if (!physical(beta + h, N, M))
                    continue;
                const int i = idx_of((long)mu + beta - nu, N, linear, M);
                if (i >= 0)
                    s += 2.0 * w * D[beta + h] * conj(D[i]);
            }
            for (int gamma = -h; gamma < N - h; ++gamma) {
                if (!physical(gamma + h, N, M))
                    continue;
                const int i = idx_of((long)mu + nu - gamma, N, linear, M);
                if (i >= 0)
                    s += conj(w) * D[i] * D[gamma + h];
            }
        }
        Dbar[nu + h] = s;
    }
}

/* xbar += J_F(x)^H ybar for F(x) = pump + i g0_mu FWM(x); pbar += ybar at mu = 0. */
static void rhs_vjp(const model* m, const cplx* x, const cplx* ybar, cplx* xbar, cplx* pbar,
                    cplx* tmp)
{
    const int N = m->N;
    for (int i = 0; i < N; ++i)
        tmp[i] = conj(I * kerr_coef(m, i)) * ybar[i];
    fwm_vjp(N, m->linear, m->M, x, tmp, tmp + N);
    for (int i = 0; i < N; ++i)
        xbar[i] += tmp[N + i];
    *pbar += ybar[N / 2];
}

int oracle_rk4ip_grad(int N, int linear, int M, const double* kappa, const double* omega,
                      double g0, const double* g0mu, double kappa_ext, double ain_re,
                      double ain_im, double sigma, double h, long nsteps, const double* D0,
                      const double* target, double eps, double* loss, double* gD0, double* gLi,
                      double* gLr, double* gP)
{
    if (check_model(N, kappa, omega) || !D0 || !target || nsteps < 0 || !loss || M < 1 || M > N)
        return ORACLE_EINVAL;
    model m = {N, linear, M, kappa, omega, g0, kappa_ext, ain_re + I * ain_im, sigma, g0mu};
    cplx* traj = malloc(sizeof(cplx) * N * (size_t)(nsteps + 1));
    cplx* w = malloc(sizeof(cplx) * 24 * N);
    cplx *E = w, *y1 = w + N, *k1 = w + 2 * N, *k2 = w + 3 * N, *k3 = w + 4 * N,
         *k4 = w + 5 * N, *u = w + 6 * N, *x2 = w + 7 * N, *x3 = w + 8 * N, *v = w + 9 * N,
         *x4 = w + 10 * N, *ww = w + 11 * N, *Db = w + 12 * N, *Dp = w + 13 * N,
         *wb = w + 14 * N, *xb = w + 15 * N, *vb = w + 16 * N, *ub = w + 17 * N,
         *kb = w + 18 * N, *Eb = w + 19 * N, *tmp = w + 20 * N; /* tmp uses 2N */
    load(N, D0, traj);
    for (int i = 0; i < N; ++i)   /* padding modes start at zero, whatever D0 holds there */
        if (!physical(i, N, M))
            traj[i] = 0.0;
    cplx* sw = malloc(sizeof(cplx) * 8 * N);
    for (long n = 0; n < nsteps; ++n) {
        memcpy(traj + (size_t)(n + 1) * N, traj + (size_t)n * N, sizeof(cplx) * N);
        step_rk4ip(&m, h, traj + (size_t)(n + 1) * N, sw);
    }
    free(sw);
    /* loss and its seed */
    const cplx* Df = traj + (size_t)nsteps * N;
    double L = 0.0;
    for (int i = 0; i < N; ++i) {
        const double P = creal(Df[i]) * creal(Df[i]) + cimag(Df[i]) * cimag(Df[i]);
        const double r = log10(P + eps) - target[i];
        L += r * r;
        const double dLdP = 2.0 * r / ((P + eps) * log(10.0));
        Db[i] = 2.0 * dLdP * Df[i];
    }
    *loss = L;
    for (int i = 0; i < N; ++i) {
        E[i] = cexp(lin_coef(&m, i) * (0.5 * h));
        gLi[i] = 0.0;
        gLr[i] = 0.0;
    }
    cplx pbar = 0.0;
    for (long n = nsteps - 1; n >= 0; --n) {
        const cplx* D = traj + (size_t)n * N;
        /* forward stages of step n */
        rhs_nonlinear(&m, D, y1);
        for (int i = 0; i < N; ++i) {
            k1[i] = E[i] * y1[i];
            u[i] = E[i] * D[i];
            x2[i] = u[i] + 0.5 * h * k1[i];
        }
        rhs_nonlinear(&m, x2, k2);
        for (int i = 0; i < N; ++i)
            x3[i] = u[i] + 0.5 * h * k2[i];
        rhs_nonlinear(&m, x3, k3);
        for (int i = 0; i < N; ++i) {
            v[i] = u[i] + h * k3[i];
            x4[i] = E[i] * v[i];
            ww[i] = u[i] + h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i]);
        }
        (void)k4;
        /* reverse: Db holds the cotangent of D_{n+1} */
        for (int i = 0; i < N; ++i) {
            wb[i] = conj(E[i]) * Db[i];
            Eb[i] = conj(ww[i]) * Db[i];
            kb[i] = h / 6.0 * Db[i]; /* k4bar */
            xb[i] = 0.0;
        }
        rhs_vjp(&m, x4, kb, xb, &pbar, tmp); /* xb = x4bar */
        for (int i = 0; i < N; ++i) {
            vb[i] = conj(E[i]) * xb[i];
            Eb[i] += conj(v[i]) * xb[i];
            ub[i] = wb[i] + vb[i];
            kb[i] = h / 3.0 * wb[i] + h * vb[i]; /* k3bar */
            xb[i] = 0.0;
        }
        rhs_vjp(&m, x3, kb, xb, &pbar, tmp); /* x3bar */
        for (int i = 0; i < N; ++i) {
            ub[i] += xb[i];
            kb[i] = h / 3.0 * wb[i] + 0.5 * h * xb[i]; /* k2bar */
            xb[i] = 0.0;
        }
        rhs_vjp(&m, x2, kb, xb, &pbar, tmp); /* x2bar */
        for (int i = 0; i < N; ++i) {
            ub[i] += xb[i];
            kb[i] = h / 6.0 * wb[i] + 0.5 * h * xb[i]; /* k1bar */
            Dp[i] = conj(E[i]) * ub[i];
            Eb[i] += conj(D[i]) * ub[i];
            xb[i] = conj(E[i]) * kb[i]; /* y1bar */
            Eb[i] += conj(y1[i]) * kb[i];
        }
        rhs_vjp(&m, D, xb, Dp, &pbar, tmp);
        for (int i = 0; i < N; ++i) {
            /* E = exp(L h/2): Lbar = conj(h/2 E) Ebar */
            const cplx Lb = conj(0.5 * h * E[i]) * Eb[i];
            gLr[i] += creal(Lb);
            gLi[i] += cimag(Lb);
            Db[i] = Dp[i];
        }
    }
    for (int i = 0; i < N; ++i)   /* D0 at the padding modes is overwritten by zero */
        if (!physical(i, N, M))
            Db[i] = 0.0;
    store(N, Db, gD0);
    gP[0] = creal(pbar);
    gP[1] = cimag(pbar);
    free(traj);
    free(w);
    return ORACLE_OK;
}

/* Loss of the forward RK4IP run alone (for finite differences). */
int oracle_rk4ip_loss(int N, int linear, int M, const double* kappa, const double* omega,
                      double g0, const double* g0mu, double kappa_ext, double ain_re,
                      double ain_im, double sigma,
                      double h, long nsteps, const double* D0, const double* target, double eps,
                      double* loss)
{
    if (check_model(N, kappa, omega) || !D0 || !target || !loss)
        return ORACLE_EINVAL;
    double* d = malloc(sizeof(double) * 2 * N);
    memcpy(d, D0, sizeof(double) * 2 * N);
    int rc = oracle_integrate(0, N, linear, M, kappa, omega, g0, g0mu, kappa_ext, ain_re, ain_im,
                              sigma,
                              h, nsteps, d);
    double L = 0.0;
    for (int i = 0; i < N; ++i) {
        const double P = d[2 * i] * d[2 * i] + d[2 * i + 1] * d[2 * i + 1];
        const double r = log10(P + eps) - target[i];
        L += r * r;
    }
    *loss = L;
    free(d);
    return rc;
}

/* ---------------------------------------------------------------------------------------
 * Discrete adjoint of the Strang split step (reverse mode through exactly the sub-steps of
 * step_strang), for the same log-power-spectrum loss and the same outputs as
 * oracle_rk4ip_grad.  One step is
 *     D1 = e D + c delta_{mu,0}             (exact linear + pump flow over dt = h/2,
 *                                            e = exp(L dt), c = phi(L_0) p, phi(L) = (e^{L dt} - 1)/L)
 *     a  = IDFT(D1),  b_j = a_j u_j,  u_j = exp(i g0 h |a_j|^2)     (exact Kerr flow)
 *     D2 = m * DFT(b) / N                   (m: physical modes)
 *     D3 = e D2 + c delta_{mu,0}.
 * Reverse, with the cotangent convention of oracle_rk4ip_grad:
 *   linear flow y = e x + c:   xbar = conj(e) ybar,  ebar += conj(x) ybar,  cbar += ybar_0;
 *   D2 = m DFT(b)/N:           bbar = IDFT(m D2bar) / N   (the adjoint of DFT is IDFT);
 *   b = a u(|a|^2), d b = u (1 + i g |a|^2) d a + i g a^2 u d conj(a):
 *                              abar = conj(u) (1 - i g |a|^2) bbar + i g a^2 u conj(bbar);
 *   a = IDFT(D1):              D1bar = DFT(abar);
 *   e = exp(L dt):             Lbar += conj(dt e) ebar;
 *   c = phi(L_0) p:            pbar = conj(phi(L_0)) cbar_total,
 *                              Lbar_0 += conj(p phi'(L_0)) cbar_total,
 *                              phi'(L) = (dt e^{L dt} - phi(L)) / L   (dt^2 / 2 at L = 0).
 * ------------------------------------------------------------------------------------- */
int oracle_strang_grad(int N, int M, const double* kappa, const double* omega, double g0,
                       double kappa_ext, double ain_re, double ain_im, double sigma, double h,
                       long nsteps, const double* D0, const double* target, double eps,
                       double* loss, double* gD0, double* gLi, double* gLr, double* gP)
{
    if (check_model(N, kappa, omega) || !D0 || !target || nsteps < 0 || !loss || M < 1 || M > N)
        return ORACLE_EINVAL;
    model m = {N, 0, M, kappa, omega, g0, kappa_ext, ain_re + I * ain_im, sigma};
    const double dt = 0.5 * h, gam = g0 * h;
    cplx* traj = malloc(sizeof(cplx) * N * (size_t)(nsteps + 1));
    cplx* w = malloc(sizeof(cplx) * 10 * N);
    cplx *e = w, *D1 = w + N, *a = w + 2 * N, *u = w + 3 * N, *D2 = w + 4 * N,
         *Db = w + 5 * N, *ab = w + 6 * N, *bb = w + 7 * N, *Eb = w + 8 * N, *tmp = w + 9 * N;
    load(N, D0, traj);
    for (int i = 0; i < N; ++i)   /* padding modes start at zero, whatever D0 holds there */
        if (!physical(i, N, M))
            traj[i] = 0.0;
    for (long n = 0; n < nsteps; ++n) {
        memcpy(traj + (size_t)(n + 1) * N, traj + (size_t)n * N, sizeof(cplx) * N);
        step_strang(&m, h, traj + (size_t)(n + 1) * N, tmp);
    }
    /* loss and its seed */
    const cplx* Df = traj + (size_t)nsteps * N;
    double L = 0.0;
    for (int i = 0; i < N; ++i) {
        const double P = creal(Df[i]) * creal(Df[i]) + cimag(Df[i]) * cimag(Df[i]);
        const double r = log10(P + eps) - target[i];
        L += r * r;
        const double dLdP = 2.0 * r / (log(10.0) * (P + eps));
        Db[i] = 2.0 * dLdP * Df[i];
    }
    *loss = L;
    const int c0 = N / 2;   /* centred index of the pumped mode mu = 0 */
    const cplx p = sqrt(kappa_ext) * m.A_in;
    for (int i = 0; i < N; ++i) {
        e[i] = cexp(lin_coef(&m, i) * dt);
        Eb[i] = 0.0;
    }
    const cplx L0 = lin_coef(&m, c0);
    const cplx phi = cabs(L0) == 0.0 ? dt : (e[c0] - 1.0) / L0;
    const cplx dphi = cabs(L0) == 0.0 ? 0.5 * dt * dt : (dt * e[c0] - phi) / L0;
    cplx cbar = 0.0;
    for (long n = nsteps - 1; n >= 0; --n) {
        const cplx* D = traj + (size_t)n * N;
        /* forward sub-steps of step n */
        for (int i = 0; i < N; ++i)
            D1[i] = e[i] * D[i];
        D1[c0] += phi * p;
        dft_modes_to_time(N, D1, a);
        for (int j = 0; j < N; ++j) {
            const double p2 = creal(a[j]) * creal(a[j]) + cimag(a[j]) * cimag(a[j]);
            u[j] = cexp(I * (gam * p2));
            tmp[j] = a[j] * u[j];
        }
        dft_time_to_modes(N, tmp, D2);
        for (int i = 0; i < N; ++i)
            D2[i] = physical(i, N, M) ? D2[i] / (double)N : 0.0;
        /* reverse; Db holds the cotangent of D3 = e D2 + c */
        cbar += Db[c0];
        for (int i = 0; i < N; ++i) {
            Eb[i] += conj(D2[i]) * Db[i];
            Db[i] = conj(e[i]) * Db[i];                          /* D2bar */
        }
        for (int i = 0; i < N; ++i)
            tmp[i] = physical(i, N, M) ? Db[i] : 0.0;
        dft_modes_to_time(N, tmp, bb);                           /* N bbar */
        for (int j = 0; j < N; ++j) {
            bb[j] /= (double)N;
            const double p2 = creal(a[j]) * creal(a[j]) + cimag(a[j]) * cimag(a[j]);
            ab[j] = conj(u[j]) * (1.0 - I * gam * p2) * bb[j] +
                    I * gam * a[j] * a[j] * u[j] * conj(bb[j]);
        }
        dft_time_to_modes(N, ab, D1);                            /* D1bar */
        cbar += D1[c0];
        for (int i = 0; i < N; ++i) {
            Eb[i] += conj(D[i]) * D1[i];
            Db[i] = conj(e[i]) * D1[i];                          /* Dbar of step n */
        }
    }
    for (int i = 0; i < N; ++i) {
        cplx Lb = conj(dt * e[i]) * Eb[i];
        if (i == c0)
            Lb += conj(p * dphi) * cbar;
        gLr[i] = creal(Lb);
        gLi[i] = cimag(Lb);
    }
    for (int i = 0; i < N; ++i)   /* D0 at the padding modes is overwritten by zero */
        if (!physical(i, N, M))
            Db[i] = 0.0;
    store(N, Db, gD0);
    const cplx pbar = conj(phi) * cbar;
    gP[0] = creal(pbar);
    gP[1] = cimag(pbar);
    free(traj);
    free(w);
    return ORACLE_OK;
}

/* Loss of the forward run alone (for finite differences): method 0 = RK4IP, 1 = Strang. */
int oracle_loss(int method, int N, int M, const double* kappa, const double* omega, double g0,
                const double* g0mu, double kappa_ext, double ain_re, double ain_im, double sigma,
                double h,
                long nsteps, const double* D0, const double* target, double eps, double* loss)
{
    if (check_model(N, kappa, omega) || !D0 || !target || !loss || (method != 0 && method != 1))
        return ORACLE_EINVAL;
    double* d = malloc(sizeof(double) * 2 * N);
    memcpy(d, D0, sizeof(double) * 2 * N);
    int rc = oracle_integrate(method, N, 0, M, kappa, omega, g0, g0mu, kappa_ext, ain_re, ain_im,
                              sigma,
                              h, nsteps, d);
    double L = 0.0;
    for (int i = 0; i < N; ++i) {
        const double P = d[2 * i] * d[2 * i] + d[2 * i + 1] * d[2 * i + 1];
        const double r = log10(P + eps) - target[i];
        L += r * r;
    }
    *loss = L;
    free(d);
    return rc;
}

/* J^H w for the FWM map at D (exposed for the dot-product test). */
int oracle_fwm_vjp(int N, int linear, int M, const double* D, const double* Wbar, double* Dbar)
{
    if (N < 1 || M < 1 || M > N || !D || !Wbar || !Dbar)
        return ORACLE_EINVAL;
    cplx* d = malloc(sizeof(cplx) * 3 * N);
    load(N, D, d);
    load(N, Wbar, d + N);
    fwm_vjp(N, linear, M, d, d + N, d + 2 * N);
    store(N, d + 2 * N, Dbar);
    free(d);
    return ORACLE_OK;
}
