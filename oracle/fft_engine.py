"""FP64 numpy engine of the CPU oracle: the same RK4IP / Strang / RK4 steps as the direct C
engine, with the four-wave-mixing sum evaluated through Eq. 4 (numpy.fft as a library
primitive).  TEST INFRASTRUCTURE ONLY.

Used where the O(N^3) direct sum is infeasible (long horizons, N >= 512).  The tests pin it
to the direct engine on every path it offers.

Arrays are (B, N) complex128 in centred order (index i <-> mu = i - N/2); all instances in a
call share N.
"""
from __future__ import annotations

import numpy as np


def _to_fft(D):
    return np.fft.ifftshift(D, axes=-1)       # centred -> mu mod N


def _to_centred(X):
    return np.fft.fftshift(X, axes=-1)        # mu mod N -> centred


def fwm(D, linear: bool = False):
    """Eq. 4: FWM_mu = (1/M) sum_j |a_j|^2 a_j exp(-2 pi i j mu / M) with
    a_j = sum_mu D_mu exp(+2 pi i j mu / M).  M = N (circular) or 2N (linear: zero padding
    to 2N removes all wrap-around because alpha - beta + gamma spans [-3N/2, 3N/2 - 3])."""
    D = np.atleast_2d(np.asarray(D, dtype=np.complex128))
    N = D.shape[-1]
    if not linear:
        a = np.fft.ifft(_to_fft(D), axis=-1) * N
        return _to_centred(np.fft.fft(np.abs(a) ** 2 * a, axis=-1) / N)
    M = 2 * N
    X = np.zeros(D.shape[:-1] + (M,), dtype=np.complex128)
    mu = np.arange(N) - N // 2
    X[..., mu % M] = D
    a = np.fft.ifft(X, axis=-1) * M
    Y = np.fft.fft(np.abs(a) ** 2 * a, axis=-1) / M
    return Y[..., mu % M]


def physical_mask(N: int, M: int) -> np.ndarray:
    """True on the M centred physical modes, mu = -floor(M/2) .. M - floor(M/2) - 1."""
    first = N // 2 - M // 2
    m = np.zeros(N, dtype=bool)
    m[first:first + M] = True
    return m


class Batch:
    """Per-instance parameters stacked for vectorised stepping.  Instances may carry M, their
    physical mode count: the other modes are held at zero and their FWM term is dropped."""

    def __init__(self, instances):
        self.N = instances[0].N
        assert all(i.N == self.N for i in instances)
        self.mask = np.stack([physical_mask(self.N, getattr(i, "M", None) or self.N)
                              for i in instances])
        self.kappa = np.stack([np.asarray(i.kappa, dtype=np.float64) for i in instances])
        self.omega = np.stack([np.asarray(i.omega, dtype=np.float64) for i in instances])
        # Kerr coefficient of each output mode: g0, or the instance's per-mode g0_mu
        self.g0 = np.stack([np.full(self.N, float(i.g0)) if getattr(i, "g0_mu", None) is None
                            else np.asarray(i.g0_mu, dtype=np.float64) for i in instances])
        self.kerr_per_mode = any(getattr(i, "g0_mu", None) is not None for i in instances)
        self.pump = np.array([np.sqrt(i.kappa_ext) * complex(i.A_in) for i in instances])
        self.sigma = np.array([i.sigma for i in instances])[:, None]
        om0 = self.omega[:, self.N // 2][:, None]
        self.L = -0.5 * self.kappa + 1j * (self.omega - om0 - self.sigma)
        self.D0 = np.where(self.mask, np.stack([np.asarray(i.D0, dtype=np.complex128)
                                                for i in instances]), 0.0)

    def F(self, D, linear=False):
        out = 1j * self.g0 * fwm(np.where(self.mask, D, 0.0), linear)
        out = np.where(self.mask, out, 0.0)
        out[:, self.N // 2] += self.pump
        return out


def rk4ip(batch: Batch, h: float, nsteps: int, D=None, linear: bool = False):
    """RK4IP (Hult 2007), E = exp(L h/2), same algebra as the direct engine."""
    D = np.where(batch.mask, batch.D0 if D is None else np.asarray(D), 0.0).astype(np.complex128)
    E = np.exp(batch.L * (0.5 * h))
    for _ in range(nsteps):
        AI = E * D
        k1 = E * batch.F(D, linear)
        k2 = batch.F(AI + 0.5 * h * k1, linear)
        k3 = batch.F(AI + 0.5 * h * k2, linear)
        k4 = batch.F(E * (AI + h * k3), linear)
        D = E * (AI + h / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3)) + h / 6.0 * k4
    return D


def strang(batch: Batch, h: float, nsteps: int, D=None):
    """Strang split step: exact linear+pump half step, exact Kerr phase rotation of the
    time-domain field a (da/dtau = i g0 |a|^2 a) followed by zeroing the padding modes, exact
    linear+pump half step."""
    if batch.kerr_per_mode:
        raise ValueError("the Strang step has no exact Kerr flow with per-mode coefficients")
    D = np.where(batch.mask, batch.D0 if D is None else np.asarray(D), 0.0).astype(np.complex128)
    N = batch.N
    e = np.exp(batch.L * (0.5 * h))
    L0 = batch.L[:, N // 2]
    c0 = np.where(np.abs(L0) > 0, (e[:, N // 2] - 1.0) / np.where(L0 == 0, 1.0, L0), 0.5 * h)
    c0 = c0 * batch.pump
    for _ in range(nsteps):
        D = e * D
        D[:, N // 2] += c0
        a = np.fft.ifft(_to_fft(D), axis=-1) * N
        a = a * np.exp(1j * batch.g0[:, :1] * np.abs(a) ** 2 * h)
        D = np.where(batch.mask, _to_centred(np.fft.fft(a, axis=-1) / N), 0.0)
        D = e * D
        D[:, N // 2] += c0
    return D


def rk4ip_one(job):
    """One instance's RK4IP run, job = (instance, h, nsteps): the unit of work the tests hand
    to a spawn process pool when many long single-instance runs are needed."""
    inst, h, nsteps = job
    return rk4ip(Batch([inst]), h, nsteps)[0]
