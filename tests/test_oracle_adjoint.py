"""Pins of the oracle's discrete adjoint (RK4IP, log-power-spectrum loss): the four-wave-mixing
VJP passes the dot-product test against finite-difference JVPs of the direct sum, and the
parameter / initial-field gradients match central finite differences of the oracle's own loss.
CPU only."""
import copy

import numpy as np
import pytest

import oracle
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
