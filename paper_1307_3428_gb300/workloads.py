"""Seeded synthetic workloads for the coupled-mode-equation (CME) integrator.

This module only builds inputs: per-mode parameter arrays, pump/detuning values and
initial fields.  It contains none of the integrator's arithmetic and is shared by the
CUDA path (tests, bench) and by the CPU oracle (tests).

Conventions (the paper's Eq. 1 and its mode label mu):
  * modes are stored in centred order: array index i <-> mode mu = i - N/2;
  * omega_mu is the cold-cavity resonance offset from the pumped mode,
    omega_mu = D2 mu^2/2 + D3 mu^3/6 (so omega_0 = 0);
  * kappa_mu is the total loss of mode mu, kappa_ext the coupling loss, g0 the Kerr
    coefficient, A_in the pump amplitude on mu = 0 and sigma the pump detuning.

Initial fields are the lower-branch continuous-wave (CW) state of the pumped mode plus
complex Gaussian noise: Re and Im are i.i.d. N(0, s^2/2), so E|z|^2 = s^2 on every mode.
The CW amplitude is the smallest positive root P of
    P [(sigma - g0 P)^2 + kappa_0^2/4] = kappa_ext |A_in|^2
(single-mode stationary point of Eq. 1 in the frame rotating with the pump), with
D_0 = sqrt(kappa_ext) A_in / (kappa_0/2 + i (sigma - g0 P)).

Seeds: noise of instance b in workload c uses numpy PCG64 seed 1307 + 1000 c + b;
random per-instance parameters of workload c use seed 1307 + 1000 c + 500.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np


@dataclasses.dataclass
class Instance:
    """One CME problem: parameters plus the initial field (centred order, complex128)."""

    N: int
    kappa: np.ndarray       # (N,) float64, total loss per mode
    omega: np.ndarray       # (N,) float64, resonance offsets omega_mu
    g0: float
    kappa_ext: float
    A_in: complex
    sigma: float
    D0: np.ndarray          # (N,) complex128 initial field
    M: Optional[int] = None  # physical modes (the centred M of the N); None: all N
    g0_mu: Optional[np.ndarray] = None  # per-mode Kerr coefficients (centred); None: g0

    @property
    def mu(self) -> np.ndarray:
        return np.arange(self.N) - self.N // 2


@dataclasses.dataclass
class Workload:
    name: str
    instances: List[Instance]
    h: float
    nsteps: int
    description: str = ""

    @property
    def mode_steps(self) -> int:
        return sum(inst.N for inst in self.instances) * self.nsteps


def dispersion(N: int, D2: float, D3: float = 0.0) -> np.ndarray:
    """omega_mu = D2 mu^2/2 + D3 mu^3/6 on the centred mode grid."""
    mu = (np.arange(N) - N // 2).astype(np.float64)
    return D2 * mu * mu / 2.0 + D3 * mu * mu * mu / 6.0


def cw_lower_branch(sigma: float, A_in: complex, kappa0: float, kappa_ext: float, g0: float) -> complex:
    """Lower-branch CW amplitude of the pumped mode (see module docstring)."""
    F2 = kappa_ext * abs(A_in) ** 2
    if g0 == 0.0:
        return np.sqrt(kappa_ext) * A_in / (kappa0 / 2 + 1j * sigma)
    coeffs = [g0 * g0, -2.0 * sigma * g0, sigma * sigma + kappa0 * kappa0 / 4.0, -F2]
    roots = np.roots(coeffs)
    real = sorted(r.real for r in roots if abs(r.imag) < 1e-9 * max(1.0, abs(r)) and r.real > 0)
    P = real[0]
    for _ in range(50):  # Newton polish in float64
        f = P * ((sigma - g0 * P) ** 2 + kappa0 * kappa0 / 4.0) - F2
        df = (sigma - g0 * P) ** 2 + kappa0 * kappa0 / 4.0 - 2.0 * g0 * P * (sigma - g0 * P)
        step = f / df
        P -= step
        if abs(step) <= 1e-17 * max(1.0, P):
            break
    return complex(np.sqrt(kappa_ext) * A_in / (kappa0 / 2 + 1j * (sigma - g0 * P)))


def _noise(N: int, s: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((N, 2)) * (s / np.sqrt(2.0))
    return z[:, 0] + 1j * z[:, 1]


def make_instance(N: int, D2: float, D3: float, sigma: float, A_in: complex, noise: float,
                  seed: int, kappa: float = 1.0, kappa_ext: float = 0.5, g0: float = 1.0,
                  cw: bool = True) -> Instance:
    kap = np.full(N, float(kappa))
    om = dispersion(N, D2, D3)
    D0 = _noise(N, noise, seed)
    if cw:
        D0[N // 2] += cw_lower_branch(sigma, A_in, kappa, kappa_ext, g0)
    return Instance(N=N, kappa=kap, omega=om, g0=float(g0), kappa_ext=float(kappa_ext),
                    A_in=complex(A_in), sigma=float(sigma), D0=D0.astype(np.complex128))


# --------------------------------------------------------------------------------------
# The synthetic workloads.  Readings for parameters the workload list leaves open:
# kappa_mu = 1, kappa_ext = 0.5, g0 = 1 wherever not stated.
# --------------------------------------------------------------------------------------

def plain64(nsteps: int = 2000) -> Workload:
    """N=64, one instance, D2=0.04, sigma=2.5, A_in=2, noise 1e-4, h=1e-3, 2000 steps."""
    inst = make_instance(64, 0.04, 0.0, 2.5, 2.0, 1e-4, seed=1307 + 1000 * 1 + 0)
    return Workload("plain_n64", [inst], 1e-3, nsteps,
                    "N=64, 1 instance, FP64, D2=0.04, sigma=2.5, A_in=2, h=1e-3")


def sweep512(n_inst: int = 256, nsteps: int = 20000, N: int = 512,
             indices: Optional[Sequence[int]] = None, seed_offset: int = 0) -> Workload:
    """N=512 x 256 instances, sigma swept linearly -2..10, A_in=2.5, D2=0.02, noise 1e-6,
    h=5e-4, 20000 steps.  `indices` selects a subset of the full 256-instance sweep (the
    selected instances keep their sweep parameters and seeds).  `seed_offset` shifts the noise
    seeds (another replica of the sweep with independent noise)."""
    full = 256
    idx = list(range(n_inst)) if indices is None else list(indices)
    insts = []
    for b in idx:
        sigma = -2.0 + 12.0 * b / (full - 1)
        insts.append(make_instance(N, 0.02, 0.0, sigma, 2.5, 1e-6,
                                   seed=1307 + 1000 * 2 + b + seed_offset))
    return Workload("sweep_n512_b256" if indices is None and n_inst == 256 else "sweep_n512_subset",
                    insts, 5e-4, nsteps,
                    "N=512, sigma in [-2,10], A_in=2.5, D2=0.02, h=5e-4")


def uneven(per_size: int = 64, nsteps: int = 50000, sizes: Sequence[int] = (256, 1024, 2048, 4096),
           indices: Optional[Sequence[int]] = None) -> Workload:
    """N in {256,1024,2048,4096} x 64 each; D2=0.01, D3=1e-4; A_in ~ U[1.5,3], sigma ~ U[0,8];
    noise 1e-6, h=2e-4, 50000 steps."""
    rng = np.random.default_rng(1307 + 1000 * 3 + 500)
    total = len(sizes) * 64
    A = rng.uniform(1.5, 3.0, total)
    S = rng.uniform(0.0, 8.0, total)
    insts = []
    b = 0
    for si, N in enumerate(sizes):
        for k in range(64):
            if k < per_size and (indices is None or b in indices):
                insts.append(make_instance(N, 0.01, 1e-4, S[b], A[b], 1e-6, seed=1307 + 1000 * 3 + b))
            b += 1
    return Workload("uneven_n256_4096", insts, 2e-4, nsteps,
                    "N in {256,1024,2048,4096} x 64, D2=0.01, D3=1e-4, h=2e-4")


def adjoint4096(batch: int = 16, nsteps: int = 10000, N: int = 4096) -> Workload:
    """N=4096 x 16: sigma ~ U[0,8], A_in ~ U[1.5,3], D2=0.01, D3=1e-4, noise 1e-6, h=2e-4."""
    rng = np.random.default_rng(1307 + 1000 * 4 + 500)
    A = rng.uniform(1.5, 3.0, batch)
    S = rng.uniform(0.0, 8.0, batch)
    insts = [make_instance(N, 0.01, 1e-4, S[b], A[b], 1e-6, seed=1307 + 1000 * 4 + b)
             for b in range(batch)]
    return Workload("adjoint_n4096_b16", insts, 2e-4, nsteps,
                    "N=4096 x 16, D2=0.01, D3=1e-4, h=2e-4")


def sech2_target(N: int, batch: int) -> np.ndarray:
    """Seeded log10 power-spectrum targets T_mu = log10(P_t sech^2(mu/W) + 1e-20),
    P_t ~ U[0.01, 1], W ~ U[N/64, N/8]; shape (batch, N), centred order."""
    rng = np.random.default_rng(1307 + 1000 * 4 + 501)
    Pt = rng.uniform(0.01, 1.0, batch)
    W = rng.uniform(N / 64.0, N / 8.0, batch)
    mu = (np.arange(N) - N // 2).astype(np.float64)
    out = np.empty((batch, N))
    for b in range(batch):
        out[b] = np.log10(Pt[b] / np.cosh(mu / W[b]) ** 2 + 1e-20)
    return out


def fig1(f0_over_sqrt2: Sequence[float] = (1.01, 1.2, 1.8, 4.0), N: int = 256, M: int = 201,
         nsteps: int = 32768, noise: float = 1e-4) -> Workload:
    """Sec. 2, Fig. 1: the normalised Eq. 2 with N = 256 (201 physical modes zero padded to
    2^8), Omega_mu = -0.00625 mu^2, kappa_mu = kappa_0, f0 = {1.01, 1.2, 1.8, 4} sqrt(2),
    tau~ = 128 pi, split step.

    Eq. 2 is the library's model with tau = tau~, kappa_mu = 2 (so -kappa_mu/2 = -1),
    g0 = 1, sqrt(kappa_ext) A_in = f0 (kappa_ext = 1) and omega_mu - omega_0 - sigma = Omega_mu;
    Omega_0 = 0 makes sigma = 0 with omega_mu = Omega_mu.  The paper states neither the step
    nor the initial field: h = 128 pi / nsteps, and the stationary CW state of the pumped mode
    (unique at zero detuning) plus seeded noise of RMS `noise` on every physical mode."""
    mu = (np.arange(N) - N // 2).astype(np.float64)
    om = -0.00625 * mu * mu
    insts = []
    for b, f in enumerate(f0_over_sqrt2):
        f0 = float(f) * np.sqrt(2.0)
        D0 = _noise(N, noise, seed=1307 + 1000 * 6 + b)
        D0[N // 2] += cw_lower_branch(0.0, f0, 2.0, 1.0, 1.0)
        insts.append(Instance(N=N, kappa=np.full(N, 2.0), omega=om.copy(), g0=1.0,
                              kappa_ext=1.0, A_in=complex(f0), sigma=0.0,
                              D0=D0.astype(np.complex128), M=M))
    return Workload("fig1_n256_m201", insts, 128.0 * np.pi / nsteps, nsteps,
                    "Fig. 1: N=256 (201 physical), Omega=-0.00625 mu^2, f0=(1.01,1.2,1.8,4)sqrt2, "
                    "tau~=128 pi, Strang")


def lle_instance(N: int, alpha: float, beta: float, F: complex, noise: float, seed: int,
                 cw: bool = True) -> Instance:
    """The normalised Lugiato-Lefever equation
        d psi/d tau = -(1 + i alpha) psi + i |psi|^2 psi - i (beta/2) d^2 psi/d theta^2 + F
    as a CME instance: psi(theta) = sum_mu A_mu exp(i mu theta) turns it into Eq. 2 with
    kappa_mu = kappa_0, Omega_mu = -alpha + (beta/2) mu^2 and f0 = F, i.e. the library's model
    with kappa_mu = 2, g0 = 1, kappa_ext = 1, A_in = F, omega_mu = (beta/2) mu^2 and
    sigma = alpha.  Initial modes: the homogeneous stationary state (the lower CW branch) plus
    seeded noise of RMS `noise` on every mode."""
    mu = (np.arange(N) - N // 2).astype(np.float64)
    D0 = _noise(N, noise, seed)
    if cw:
        D0[N // 2] += cw_lower_branch(alpha, F, 2.0, 1.0, 1.0)
    return Instance(N=N, kappa=np.full(N, 2.0), omega=0.5 * beta * mu * mu, g0=1.0,
                    kappa_ext=1.0, A_in=complex(F), sigma=float(alpha),
                    D0=D0.astype(np.complex128))


def octave(N: int = 1 << 17, nsteps: int = 10000) -> Workload:
    """N=2^17 single instance: D2=2e-4, D3=-4e-7, sigma=4, A_in=3, noise 1e-8, h=1e-4."""
    inst = make_instance(N, 2e-4, -4e-7, 4.0, 3.0, 1e-8, seed=1307 + 1000 * 5 + 0)
    return Workload("octave_n131072", [inst], 1e-4, nsteps,
                    "N=2^17, D2=2e-4, D3=-4e-7, sigma=4, A_in=3, h=1e-4")


def random_instance(N: int, seed: int, g0: float = 1.0, kappa: float = 1.0, amp: float = 0.5,
                    D2: float = 0.02, sigma: float = 1.0, A_in: complex = 1.5,
                    kappa_ext: float = 0.5) -> Instance:
    """A generic test instance: random complex field of RMS amplitude `amp` on all modes,
    per-mode loss jittered around `kappa`."""
    rng = np.random.default_rng(seed)
    D0 = (rng.standard_normal(N) + 1j * rng.standard_normal(N)) * (amp / np.sqrt(2.0))
    kap = kappa * (1.0 + 0.1 * rng.uniform(-1, 1, N)) if kappa != 0.0 else np.zeros(N)
    om = dispersion(N, D2, 0.0)
    return Instance(N=N, kappa=kap, omega=om, g0=float(g0), kappa_ext=float(kappa_ext),
                    A_in=complex(A_in), sigma=float(sigma), D0=D0)


def kerr_slope(g0: float, N: int, slope: float) -> np.ndarray:
    """A frequency-dependent Kerr coefficient, linear across the band:
    g0_mu = g0 (1 + slope mu / (N/2)) on the centred mode grid (the nonlinear coefficient
    scales with the mode frequency and the inverse effective area, both smooth in mu)."""
    mu = (np.arange(N) - N // 2).astype(np.float64)
    return g0 * (1.0 + slope * mu / (N / 2.0))
