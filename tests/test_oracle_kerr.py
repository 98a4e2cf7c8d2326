"""Pins of the oracle's per-mode Kerr coefficient g0_mu (Sec. 2: a constant g0 is no necessary
restriction of the coupled mode equations, and frequency-dependent coefficients fit them easily).
Read here as the coefficient of the output mode's four-wave-mixing term,
    F_mu(D) = delta_{mu,0} sqrt(kappa_ext) A_in + i g0_mu FWM_mu(D),
the form that keeps Eq. 4 (a per-mode multiply after the forward transform).  CPU only."""
import copy

import numpy as np
import pytest

import oracle
from oracle import fft_engine
from paper_1307_3428_gb300 import workloads as wl


def test_constant_per_mode_coefficient_equals_scalar_g0():
    inst = wl.random_instance(16, 300, g0=1.3, amp=0.3)
    ref = oracle.integrate(inst, 0.01, 40, oracle.RK4IP)
    i2 = copy.deepcopy(inst)
    i2.g0_mu = np.full(16, 1.3)
    i2.g0 = 0.0           # ignored when g0_mu is given
    assert np.array_equal(oracle.integrate(i2, 0.01, 40, oracle.RK4IP), ref)


def test_two_mode_cross_phase_closed_form():
    """Only mu = 0 and mu = 1 excited (linear sum, so nothing wraps): the sum's terms are
    the self- and cross-phase terms |D0|^2 D0 + 2 |D1|^2 D0 on mu = 0, |D1|^2 D1 + 2 |D0|^2 D1
    on mu = 1, and the generated lines D1^2 conj(D0) on mu = 2 and D0^2 conj(D1) on mu = -1;
    each carries the coefficient of its own (output) mode."""
    N = 8
    c = N // 2
    D = np.zeros(N, complex)
    D0, D1 = 0.7 - 0.2j, 0.3 + 0.5j
    D[c], D[c + 1] = D0, D1
    g = np.linspace(0.5, 2.2, N)
    F = oracle.rhs(D, 9.9, 0.0, 0.0, linear=True, g0_mu=g)
    exp = np.zeros(N, complex)
    exp[c] = 1j * g[c] * (abs(D0) ** 2 + 2 * abs(D1) ** 2) * D0
    exp[c + 1] = 1j * g[c + 1] * (abs(D1) ** 2 + 2 * abs(D0) ** 2) * D1
    exp[c + 2] = 1j * g[c + 2] * D1 ** 2 * np.conj(D0)
    exp[c - 1] = 1j * g[c - 1] * D0 ** 2 * np.conj(D1)
    assert np.max(np.abs(F - exp)) <= 1e-15


def test_single_mode_rotation_uses_the_pumped_modes_coefficient():
    """Lossless, unpumped, only mu = 0 excited: D_0(tau) = D_0 exp(i (g0_0 |D_0|^2 - sigma) tau)
    with the coefficient of mode 0; RK4IP within its fourth-order error."""
    N = 8
    inst = wl.make_instance(N, 0.0, 0.0, 0.4, 0.0, 0.0, seed=1, kappa=0.0, cw=False)
    inst.kappa_ext = 0.0
    inst.D0 = np.zeros(N, complex)
    inst.D0[N // 2] = 0.9 + 0.4j
    inst.g0_mu = np.linspace(0.2, 3.0, N)
    h, n = 1e-3, 500
    D = oracle.integrate(inst, h, n, oracle.RK4IP)
    g = inst.g0_mu[N // 2]
    exact = inst.D0[N // 2] * np.exp(1j * (g * abs(inst.D0[N // 2]) ** 2 - inst.sigma) * n * h)
    assert abs(D[N // 2] - exact) <= 1e-12
    assert np.max(np.abs(np.delete(D, N // 2))) == 0.0


def test_eq4_engine_matches_direct_engine_with_per_mode_coefficients():
    insts = []
    for k, N in enumerate((16, 16)):
        i = wl.random_instance(N, 310 + k, amp=0.3)
        i.g0_mu = wl.kerr_slope(1.0, N, 0.3 * (k + 1))
        insts.append(i)
    ref = [oracle.integrate(i, 0.01, 30, oracle.RK4IP) for i in insts]
    got = fft_engine.rk4ip(fft_engine.Batch(insts), 0.01, 30)
    for g, r in zip(got, ref):
        assert np.max(np.abs(g - r)) <= 1e-13 * np.max(np.abs(r))


def test_strang_refuses_per_mode_coefficients():
    i = wl.random_instance(8, 320)
    i.g0_mu = np.ones(8)
    with pytest.raises(ValueError):
        oracle.integrate(i, 0.01, 3, oracle.STRANG)
    with pytest.raises(ValueError):
        fft_engine.strang(fft_engine.Batch([i]), 0.01, 3)


def test_adjoint_with_per_mode_coefficients_matches_central_differences():
    N, h, n = 8, 0.02, 30
    inst = wl.make_instance(N, 0.05, 0.01, 1.3, 1.4 + 0.2j, 0.05, seed=330)
    inst.g0_mu = wl.kerr_slope(1.0, N, 0.4)
    T = np.log10(np.random.default_rng(331).uniform(1e-4, 0.5, N))
    g = oracle.log_spectrum_grad(inst, h, n, T)
    L0 = oracle.log_spectrum_loss(inst, h, n, T)
    assert abs(L0 - g["loss"]) <= 1e-12 * abs(L0)
    mu = np.arange(N) - N // 2

    def loss_with(**kw):
        i2 = copy.deepcopy(inst)
        for k, v in kw.items():
            setattr(i2, k, v)
        return oracle.log_spectrum_loss(i2, h, n, T)

    e = 1e-6
    checks = {"sigma": (lambda s: loss_with(sigma=inst.sigma + s), g["sigma"]),
              "D2": (lambda s: loss_with(omega=inst.omega + s * mu ** 2 / 2.0), g["D2"]),
              "A_im": (lambda s: loss_with(A_in=inst.A_in + 1j * s), g["A_in"].imag)}
    rng = np.random.default_rng(332)
    for r in range(3):
        v = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        checks[f"D0_{r}"] = (lambda s, v=v: loss_with(D0=inst.D0 + s * v),
                             float(np.real(np.vdot(g["D0"], v))))
    for name, (f, ad) in checks.items():
        fd = (8 * (f(e) - f(-e)) - (f(2 * e) - f(-2 * e))) / (12 * e)
        assert abs(fd - ad) <= 1e-6 * max(abs(fd), 1e-3 * abs(L0)), (name, fd, ad)
