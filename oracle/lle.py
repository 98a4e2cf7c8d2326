"""The Lugiato-Lefever equation (LLE) in the time domain, for the check of Sec. 2's statement
that the coupled mode equations are a discrete Fourier expansion of a driven and damped NLS
(LLE) equation.  TEST INFRASTRUCTURE ONLY.

Normalised LLE on the ring coordinate theta in [0, 2 pi), sampled at theta_j = 2 pi j / N:

    d psi/d tau = -(1 + i alpha) psi + i |psi|^2 psi - i (beta/2) d^2 psi/d theta^2 + F,

with the second derivative taken spectrally (numpy.fft as the library primitive).  Written
with psi(theta) = sum_mu A_mu exp(i mu theta), it is Eq. 2 with kappa_mu = kappa_0,
Omega_mu = -alpha + (beta/2) mu^2 and f0 = F, and psi_j is the unnormalised inverse transform
of A over the mode number.  Integrated here by classic RK4 in the time domain.
"""
from __future__ import annotations

import numpy as np


def _k(N):
    """Wavenumbers of numpy.fft's ordering (mu mod N, the upper half negative)."""
    return np.fft.fftfreq(N, d=1.0 / N)


def d2_theta(psi):
    """Spectral second derivative d^2/d theta^2 on the N-point ring."""
    N = psi.shape[-1]
    return np.fft.ifft(-(_k(N) ** 2) * np.fft.fft(psi))


def rhs(psi, alpha, beta, F):
    return (-(1.0 + 1j * alpha) * psi + 1j * np.abs(psi) ** 2 * psi
            - 1j * (beta / 2.0) * d2_theta(psi) + F)


def rk4(psi0, alpha, beta, F, h, nsteps):
    """Classic RK4 on the LLE in the time domain."""
    psi = np.asarray(psi0, dtype=np.complex128).copy()
    for _ in range(nsteps):
        k1 = rhs(psi, alpha, beta, F)
        k2 = rhs(psi + 0.5 * h * k1, alpha, beta, F)
        k3 = rhs(psi + 0.5 * h * k2, alpha, beta, F)
        k4 = rhs(psi + h * k3, alpha, beta, F)
        psi = psi + h / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    return psi


def modes_to_theta(A):
    """psi_j = sum_mu A_mu exp(2 pi i j mu / N) for a centred mode vector A."""
    N = A.shape[-1]
    return np.fft.ifft(np.fft.ifftshift(A, axes=-1), axis=-1) * N


def theta_to_modes(psi):
    """The inverse of modes_to_theta: centred A_mu = (1/N) sum_j psi_j exp(-2 pi i j mu / N)."""
    N = psi.shape[-1]
    return np.fft.fftshift(np.fft.fft(psi, axis=-1), axes=-1) / N
