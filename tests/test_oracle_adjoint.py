"""Pins of the oracle's discrete adjoints (RK4IP and the Strang split step, log-power-spectrum
loss): the four-wave-mixing VJP passes the dot-product test against finite-difference JVPs of
the direct sum, the parameter / initial-field gradients match central finite differences of the
oracle's own loss, and the Strang gradient of a linear run (g0 = 0) equals its closed form.
CPU only."""
import copy

import numpy as np
import pytest

import oracle
from oracle import fft_engine
from paper_1307_3428_gb300 import workloads as wl


def rand(N, seed, amp=0.5):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(N) + 1j * rng.standard_normal(N)) * amp


@pytest.mark.parametrize("N", [3, 4, 8, 16])
@pytest.mark.parametrize("linear", [False, True])
def test_fwm_vjp_dot_product(N, linear):
    D, v, w = rand(N, 1), rand(N, 2), rand(N, 3)
    eps = 1e-5
    jv = (oracle.fwm(D + eps * v, linear) - oracle.fwm(D - eps * v, linear)) / (2 * eps)
    lhs = np.real(np.vdot(w, jv))
    rhs = np.real(np.vdot(oracle.fwm_vjp(D, w, linear), v))
    assert abs(lhs - rhs) <= 1e-9 * max(1.0, abs(lhs))


def _instance(N, seed):
    inst = wl.make_instance(N, 0.05, 0.01, 1.3, 1.4 + 0.2j, 0.05, seed=seed)
    inst.kappa = np.full(N, 1.0)
    return inst


def _target(N, seed):
    rng = np.random.default_rng(seed)
    return np.log10(rng.uniform(1e-4, 0.5, N))


def test_gradients_match_central_differences():
    N, h, n = 8, 0.02, 40
    inst = _instance(N, 7)
    T = _target(N, 8)
    g = oracle.log_spectrum_grad(inst, h, n, T, eps=1e-20)
    L0 = oracle.log_spectrum_loss(inst, h, n, T)
    assert abs(L0 - g["loss"]) <= 1e-12 * abs(L0)
    mu = np.arange(N) - N // 2

    def loss_with(**kw):
        i2 = copy.deepcopy(inst)
        for k, v in kw.items():
            setattr(i2, k, v)
        return oracle.log_spectrum_loss(i2, h, n, T)

    e = 1e-6
    checks = {
        "sigma": (lambda s: loss_with(sigma=inst.sigma + s), g["sigma"]),
        "D2": (lambda s: loss_with(omega=inst.omega + s * mu ** 2 / 2.0), g["D2"]),
        "D3": (lambda s: loss_with(omega=inst.omega + s * mu ** 3 / 6.0), g["D3"]),
        "A_re": (lambda s: loss_with(A_in=inst.A_in + s), g["A_in"].real),
        "A_im": (lambda s: loss_with(A_in=inst.A_in + 1j * s), g["A_in"].imag),
        "kappa": (lambda s: loss_with(kappa=inst.kappa + s), float(np.sum(g["kappa"]))),
    }
    for name, (f, ad) in checks.items():
        fd = (f(e) - f(-e)) / (2 * e)
        assert abs(fd - ad) <= 1e-6 * max(abs(fd), 1e-3 * abs(L0)), (name, fd, ad)
    rng = np.random.default_rng(9)
    for _ in range(4):
        v = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        fd = (loss_with(D0=inst.D0 + e * v) - loss_with(D0=inst.D0 - e * v)) / (2 * e)
        ad = np.real(np.vdot(g["D0"], v))
        assert abs(fd - ad) <= 1e-6 * max(abs(fd), 1e-3 * abs(L0)), (fd, ad)


def test_gradient_of_omega_entries_and_linear_sum():
    N, h, n = 8, 0.02, 25
    inst = _instance(N, 11)
    T = _target(N, 12)
    for linear in (False, True):
        g = oracle.log_spectrum_grad(inst, h, n, T, linear=linear)
        e = 1e-6
        for k in (0, N // 2, N - 1):
            i1, i2 = copy.deepcopy(inst), copy.deepcopy(inst)
            i1.omega = inst.omega.copy(); i1.omega[k] += e
            i2.omega = inst.omega.copy(); i2.omega[k] -= e
            fd = (oracle.log_spectrum_loss(i1, h, n, T, linear=linear) -
                  oracle.log_spectrum_loss(i2, h, n, T, linear=linear)) / (2 * e)
            assert abs(fd - g["omega"][k]) <= 1e-6 * max(abs(fd), 1e-6), (linear, k, fd, g["omega"][k])


# ---------------------------------------------------------------------------------------------
# Discrete adjoint of the Strang split step (the split-step Fourier method of Sec. 2 with the
# field held in the frequency domain): exact linear + pump half flows around the exact Kerr
# phase rotation of the time-domain field.

def _strang_checks(inst, h, n, T, e=1e-6):
    """Central differences (fourth order) of the oracle's Strang loss against its adjoint, for
    sigma, D2, D3, A_in, kappa (all modes, and the pumped mode alone, whose loss enters the
    pump increment of the linear flow), two omega entries and three initial-field
    directions."""
    S = oracle.STRANG
    g = oracle.log_spectrum_grad(inst, h, n, T, method=S)
    L0 = oracle.log_spectrum_loss(inst, h, n, T, method=S)
    assert abs(L0 - g["loss"]) <= 1e-12 * abs(L0)
    N = inst.N
    mu = np.arange(N) - N // 2
    onehot = lambda k: (np.arange(N) == k).astype(float)

    def loss_with(**kw):
        i2 = copy.deepcopy(inst)
        for k, v in kw.items():
            setattr(i2, k, v)
        return oracle.log_spectrum_loss(i2, h, n, T, method=S)

    checks = {
        "sigma": (lambda s: loss_with(sigma=inst.sigma + s), g["sigma"]),
        "D2": (lambda s: loss_with(omega=inst.omega + s * mu ** 2 / 2.0), g["D2"]),
        "D3": (lambda s: loss_with(omega=inst.omega + s * mu ** 3 / 6.0), g["D3"]),
        "A_re": (lambda s: loss_with(A_in=inst.A_in + s), g["A_in"].real),
        "A_im": (lambda s: loss_with(A_in=inst.A_in + 1j * s), g["A_in"].imag),
        "kappa": (lambda s: loss_with(kappa=inst.kappa + s), float(np.sum(g["kappa"]))),
        "kappa_0": (lambda s: loss_with(kappa=inst.kappa + s * onehot(N // 2)),
                    g["kappa"][N // 2]),
        "omega_1": (lambda s: loss_with(omega=inst.omega + s * onehot(N // 2 + 1)),
                    g["omega"][N // 2 + 1]),
        "omega_0": (lambda s: loss_with(omega=inst.omega + s * onehot(0)), g["omega"][0]),
    }
    rng = np.random.default_rng(19)
    for r in range(3):
        v = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        checks[f"D0_{r}"] = (lambda s, v=v: loss_with(D0=inst.D0 + s * v),
                             float(np.real(np.vdot(g["D0"], v))))
    for name, (f, ad) in checks.items():
        fd = (8 * (f(e) - f(-e)) - (f(2 * e) - f(-2 * e))) / (12 * e)
        assert abs(fd - ad) <= 1e-6 * max(abs(fd), 1e-3 * abs(L0)), (name, fd, ad)
    return g


def test_strang_gradients_match_central_differences():
    N, h, n = 8, 0.02, 40
    inst = _instance(N, 7)
    _strang_checks(inst, h, n, _target(N, 8))


def test_strang_gradients_strong_kerr_phase():
    """A large Kerr phase per step (g0 |a|^2 h of order 1), where the phase-rotation factors of
    the Kerr VJP dominate, and an odd mode count."""
    N, h, n = 5, 0.15, 12
    inst = wl.make_instance(N, 0.3, 0.0, 0.7, 2.2 - 0.4j, 0.3, seed=21)
    inst.D0 = inst.D0 * 3.0
    _strang_checks(inst, h, n, _target(N, 22))


def test_strang_gradients_with_padding_modes():
    """6 physical modes in an 8-point transform: the padding modes carry no gradient."""
    N, h, n = 8, 0.02, 30
    inst = _instance(N, 31)
    inst.M = 6
    g = _strang_checks(inst, h, n, _target(N, 32))
    pad = ~fft_engine.physical_mask(N, 6)
    assert np.all(g["D0"][pad] == 0)


def test_strang_gradient_linear_limit_closed_form():
    """g0 = 0: Strang is the exact affine flow D(tau) = e^{L tau} D0 + (e^{L tau} - 1)/L p on
    the pumped mode.  The loss then has a closed-form gradient in sigma through
    dD_mu/dsigma = -i tau e^{L tau} D0_mu (+ the pump term's derivative on mu = 0)."""
    N, h, n = 4, 0.05, 20
    inst = _instance(N, 41)
    inst.g0 = 0.0
    T = _target(N, 42)
    g = oracle.log_spectrum_grad(inst, h, n, T, method=oracle.STRANG)
    tau = n * h
    L = -0.5 * inst.kappa + 1j * (inst.omega - inst.omega[N // 2] - inst.sigma)
    p = np.sqrt(inst.kappa_ext) * inst.A_in
    e = np.exp(L * tau)
    D = e * inst.D0
    dD = -1j * tau * e * inst.D0             # dL_mu/dsigma = -i
    c = N // 2
    D[c] += (e[c] - 1.0) / L[c] * p
    dD[c] += -1j * (tau * e[c] * L[c] - (e[c] - 1.0)) / L[c] ** 2 * p
    P = np.abs(D) ** 2
    r = np.log10(P + 1e-20) - T
    dL = np.sum(2 * r / ((P + 1e-20) * np.log(10)) * 2 * np.real(np.conj(D) * dD))
    assert abs(g["loss"] - np.sum(r ** 2)) <= 1e-12 * np.sum(r ** 2)
    assert abs(g["sigma"] - dL) <= 1e-9 * abs(dL)
