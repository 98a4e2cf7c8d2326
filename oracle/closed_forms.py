"""Closed-form results of the CME model, used to pin the oracle.  TEST INFRASTRUCTURE ONLY.

All formulas follow from Eq. 1 written in the frame rotating with the pump,
    dD_mu/dtau = (-kappa_mu/2 + i(omega_mu - sigma)) D_mu + delta_{mu,0} sqrt(kappa_ext) A_in
                 + i g0 sum_{alpha-beta+gamma=mu} D_alpha conj(D_beta) D_gamma,
with omega_0 = 0.
"""
from __future__ import annotations

import numpy as np


def cw_powers(sigma, A_in, kappa0, kappa_ext, g0):
    """All positive real roots P of P[(sigma - g0 P)^2 + kappa0^2/4] = kappa_ext |A_in|^2,
    sorted ascending: intracavity powers of the single-mode stationary states."""
    F2 = kappa_ext * abs(A_in) ** 2
    c = [g0 * g0, -2.0 * sigma * g0, sigma * sigma + kappa0 * kappa0 / 4.0, -F2]
    r = np.roots(c)
    out = []
    for z in r:
        if abs(z.imag) < 1e-9 * max(1.0, abs(z)) and z.real > 0:
            P = z.real
            for _ in range(60):
                f = P * ((sigma - g0 * P) ** 2 + kappa0 ** 2 / 4.0) - F2
                df = (sigma - g0 * P) ** 2 + kappa0 ** 2 / 4.0 - 2 * g0 * P * (sigma - g0 * P)
                P -= f / df
            out.append(P)
    return sorted(out)


def cw_field(P, sigma, A_in, kappa0, kappa_ext, g0):
    """Stationary pumped-mode amplitude for intracavity power P."""
    return np.sqrt(kappa_ext) * A_in / (kappa0 / 2.0 + 1j * (sigma - g0 * P))


def mi_rates(P, omega, sigma, kappa, g0):
    """Eigenvalues lambda(mu) of the linearisation about the CW state for the sideband pair
    (mu, -mu):  lambda = -kappa/2 + i(omega_mu - omega_-mu)/2 +- sqrt(g0^2 P^2 - delta^2),
    delta = (omega_mu + omega_-mu)/2 - sigma + 2 g0 P.  `omega` is a callable mu -> omega_mu.
    Returns a function of mu giving the eigenvalue with the larger real part."""
    om = omega

    def lam(mu):
        delta = (om(mu) + om(-mu)) / 2.0 - sigma + 2.0 * g0 * P
        return (-kappa / 2.0 + 1j * (om(mu) - om(-mu)) / 2.0
                + np.sqrt(complex(g0 * g0 * P * P - delta ** 2)))
    return lam


def max_mi_gain(P, N, D2, D3, sigma, kappa, g0):
    """max over sideband pairs of Re(lambda): positive means the CW state is unstable."""
    om = lambda m: D2 * m * m / 2.0 + D3 * m ** 3 / 6.0
    lam = mi_rates(P, om, sigma, kappa, g0)
    return max(lam(m).real for m in range(1, N // 2))


def single_mode(D0, sigma, g0, tau):
    """Lossless, unpumped, only mu=0 excited: D_0(tau) = D_0 exp(i(g0 |D_0|^2 - sigma) tau)."""
    return D0 * np.exp(1j * (g0 * abs(D0) ** 2 - sigma) * tau)


def linear_affine(D0, L, pump, tau):
    """g0 = 0: D(tau) = e^{L tau} D0 + (e^{L tau} - 1)/L * pump (pump only on the centre)."""
    e = np.exp(L * tau)
    out = e * D0
    N = len(D0)
    out[N // 2] += (e[N // 2] - 1.0) / L[N // 2] * pump
    return out
