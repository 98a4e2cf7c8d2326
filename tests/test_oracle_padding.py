"""Pins of the oracle's physical-mode count M (the zero padding of Sec. 2: 201 modes in a
256-point transform): of N modes only the centred M, mu = -floor(M/2) .. M - floor(M/2) - 1,
are physical; the others stay at zero and the FWM sum runs over physical modes only.

What pins it: brute-force enumeration of the constraint alpha - beta + gamma = mu (mod N)
over the physical modes; for N >= 2M no triple wraps into the band, so the padded sum equals
the oracle's linear (non-wrapping) sum of the M-mode system, and the padded integrators equal
the M-mode linear-sum integrators; the padded FWM VJP passes the dot-product test; the padded
gradient matches central differences of the padded loss.  CPU only."""
import copy
import itertools

import numpy as np
import pytest

import oracle
from oracle import fft_engine
from paper_1307_3428_gb300 import workloads as wl


def rand(N, seed, amp=0.5):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(N) + 1j * rng.standard_normal(N)) * amp


def band(N, M):
    first = N // 2 - M // 2
    return np.arange(first, first + M)


def pad(DM, N):
    """The M-mode centred vector DM placed into the band of an N-mode centred vector."""
    M = len(DM)
    out = np.zeros(N, dtype=complex)
    out[band(N, M)] = DM
    return out


def brute_padded(D, M):
    """Every (alpha, beta, gamma) of the physical modes whose alpha - beta + gamma equals a
    physical mu modulo N."""
    N = len(D)
    modes = [i - N // 2 for i in band(N, M)]
    out = np.zeros(N, dtype=complex)
    for mu in modes:
        for a, b, g in itertools.product(modes, repeat=3):
            if (a - b + g - mu) % N == 0:
                out[mu + N // 2] += D[a + N // 2] * np.conj(D[b + N // 2]) * D[g + N // 2]
    return out


@pytest.mark.parametrize("N,M", [(8, 5), (8, 6), (8, 3), (6, 5), (4, 4), (8, 1)])
def test_padded_fwm_equals_enumeration(N, M):
    """Includes N < 2M, where triples wrap into the band (as 201 modes in 256 do)."""
    D = pad(rand(M, 20 + N + M), N)
    got = oracle.fwm(D, M=M)
    ref = brute_padded(D, M)
    assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("N,M", [(16, 7), (16, 8), (32, 11), (64, 32)])
def test_padding_to_2m_is_the_linear_sum(N, M):
    DM = rand(M, 40 + M)
    got = oracle.fwm(pad(DM, N), M=M)
    lin = oracle.fwm(DM, linear=True)
    assert np.max(np.abs(got[band(N, M)] - lin)) <= 1e-12 * np.max(np.abs(lin))
    outside = np.setdiff1d(np.arange(N), band(N, M))
    assert np.all(got[outside] == 0)


def test_unpadded_mask_is_identity():
    D = rand(16, 5)
    assert np.array_equal(oracle.fwm(D, M=16), oracle.fwm(D))


def _padded_instance(M, N, seed):
    """An M-mode instance and the same problem padded to N modes (padding modes carry
    arbitrary values that the padded integrators must ignore)."""
    base = wl.random_instance(M, seed, amp=0.3, sigma=0.7, A_in=1.2 + 0.3j)
    mu_N = np.arange(N) - N // 2
    padded = copy.deepcopy(base)
    padded.N, padded.M = N, M
    padded.kappa = np.full(N, 1.0)
    padded.kappa[band(N, M)] = base.kappa
    padded.omega = 0.02 * mu_N ** 2 / 2.0
    padded.omega[band(N, M)] = base.omega
    padded.D0 = rand(N, seed + 1, amp=5.0)        # junk in the padding modes
    padded.D0[band(N, M)] = base.D0
    return base, padded


@pytest.mark.parametrize("method", [oracle.RK4IP, oracle.RK4])
@pytest.mark.parametrize("N,M", [(16, 7), (16, 8)])
def test_padded_integrators_equal_linear_m_mode_system(method, N, M):
    base, padded = _padded_instance(M, N, 60 + M)
    got = oracle.integrate(padded, 5e-3, 40, method)
    ref = oracle.integrate(base, 5e-3, 40, method, linear=True)
    assert np.max(np.abs(got[band(N, M)] - ref)) <= 1e-12 * np.max(np.abs(ref))
    outside = np.setdiff1d(np.arange(N), band(N, M))
    assert np.all(got[outside] == 0)


@pytest.mark.parametrize("N,M", [(16, 11), (32, 25), (16, 7)])
def test_padded_strang_matches_the_eq4_engine(N, M):
    """Strang has no linear-sum form in the oracle; the direct engine (naive transforms) and the
    numpy Eq. 4 engine must agree with padding, including the aliasing case N < 2M."""
    _, padded = _padded_instance(M, N, 80 + M)
    got = oracle.integrate(padded, 4e-3, 30, oracle.STRANG)
    ref = fft_engine.strang(fft_engine.Batch([padded]), 4e-3, 30)[0]
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("N,M", [(16, 11), (32, 25), (16, 7)])
def test_padded_rk4ip_direct_matches_the_eq4_engine(N, M):
    _, padded = _padded_instance(M, N, 90 + M)
    got = oracle.integrate(padded, 4e-3, 30, oracle.RK4IP)
    ref = fft_engine.rk4ip(fft_engine.Batch([padded]), 4e-3, 30)[0]
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("N,M", [(8, 5), (8, 3), (16, 11)])
def test_padded_fwm_vjp_dot_product(N, M):
    D, v, w = pad(rand(M, 1), N), rand(N, 2), rand(N, 3)
    e = 1e-5
    jv = (oracle.fwm(D + e * v, M=M) - oracle.fwm(D - e * v, M=M)) / (2 * e)
    lhs = np.real(np.vdot(w, jv))
    rhs = np.real(np.vdot(oracle.fwm_vjp(D, w, M=M), v))
    assert abs(lhs - rhs) <= 1e-9 * max(1.0, abs(lhs))


def test_padded_gradient_matches_central_differences():
    N, M, h, n = 8, 5, 0.02, 30
    _, inst = _padded_instance(M, N, 120)
    rng = np.random.default_rng(121)
    T = np.log10(rng.uniform(1e-4, 0.5, N))
    g = oracle.log_spectrum_grad(inst, h, n, T)

    def loss_with(**kw):
        i2 = copy.deepcopy(inst)
        for k, v in kw.items():
            setattr(i2, k, v)
        return oracle.log_spectrum_loss(i2, h, n, T)

    L0 = loss_with()
    e = 1e-6
    for name, f, ad in (("sigma", lambda s: loss_with(sigma=inst.sigma + s), g["sigma"]),
                        ("A_re", lambda s: loss_with(A_in=inst.A_in + s), g["A_in"].real)):
        fd = (f(e) - f(-e)) / (2 * e)
        assert abs(fd - ad) <= 1e-6 * max(abs(fd), 1e-3 * abs(L0)), (name, fd, ad)
    for k in range(3):
        v = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        fd = (loss_with(D0=inst.D0 + e * v) - loss_with(D0=inst.D0 - e * v)) / (2 * e)
        ad = np.real(np.vdot(g["D0"], v))
        assert abs(fd - ad) <= 1e-6 * max(abs(fd), 1e-3 * abs(L0)), (fd, ad)
    outside = np.setdiff1d(np.arange(N), band(N, M))
    assert np.all(g["D0"][outside] == 0)
