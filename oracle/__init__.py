"""FP64 CPU oracle for the coupled mode equations (CMEs).

TEST INFRASTRUCTURE ONLY: imported by `tests/`, by `__graft_entry__.smoke()` and by the
CPU-baseline leg of `bench.py`, never by the product package.  It shares no code with the
CUDA path.

Two engines:
  * `direct` (C library `cme_oracle.c`): the four-wave-mixing sum as the direct O(N^3)
    triple sum of Eq. 2 / Eq. 3, RK4IP / Strang / plain RK4 steps in textbook order, naive
    O(N^2) transforms over the mode number.  This is the definition.
  * `fft_engine` (numpy): the same integrators with the FWM sum evaluated through Eq. 4 using
    numpy.fft as a library primitive; used only where O(N^3) is infeasible, and pinned to the
    direct engine by the tests.

Layout: arrays hold modes in centred order, index i <-> mu = i - N/2.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libcme_oracle.so")
_SRC = os.path.join(_HERE, "cme_oracle.c")
_lock = threading.Lock()
_lib = None

RK4IP, STRANG, RK4 = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (plain -O2, no fast-math)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=gnu11", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _configure(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    c_int, c_long, c_double = ctypes.c_int, ctypes.c_long, ctypes.c_double
    lib.oracle_fwm.argtypes = [c_int, c_int, c_int, dp, dp]
    lib.oracle_rhs.argtypes = [c_int, c_int, c_int, c_double, dp, c_double, c_double, c_double,
                               dp, dp]
    lib.oracle_integrate.argtypes = [c_int, c_int, c_int, c_int, dp, dp, c_double, dp, c_double,
                                     c_double, c_double, c_double, c_double, c_long, dp]
    lib.oracle_integrate_eq1.argtypes = [c_int, c_int, dp, dp, c_double, c_double,
                                         c_double, c_double, c_double, c_double,
                                         c_double, c_long, dp]
    lib.oracle_dft.argtypes = [c_int, c_int, dp, dp]
    lib.oracle_invariants.argtypes = [c_int, c_int, dp, c_double, c_double, dp, dp]
    lib.oracle_rk4ip_grad.argtypes = [c_int, c_int, c_int, dp, dp, c_double, dp, c_double,
                                      c_double, c_double, c_double, c_double, c_long, dp, dp,
                                      c_double, dp, dp, dp, dp, dp]
    lib.oracle_rk4ip_loss.argtypes = [c_int, c_int, c_int, dp, dp, c_double, dp, c_double,
                                      c_double, c_double, c_double, c_double, c_long, dp, dp,
                                      c_double, dp]
    lib.oracle_fwm_vjp.argtypes = [c_int, c_int, c_int, dp, dp, dp]
    lib.oracle_strang_grad.argtypes = [c_int, c_int, dp, dp, c_double, c_double, c_double,
                                       c_double, c_double, c_double, c_long, dp, dp, c_double,
                                       dp, dp, dp, dp, dp]
    lib.oracle_loss.argtypes = [c_int, c_int, c_int, dp, dp, c_double, dp, c_double, c_double,
                                c_double, c_double, c_double, c_long, dp, dp, c_double, dp]
    for name in ("oracle_fwm", "oracle_rhs", "oracle_integrate", "oracle_integrate_eq1",
                 "oracle_dft", "oracle_invariants", "oracle_rk4ip_grad",
                 "oracle_rk4ip_loss", "oracle_fwm_vjp", "oracle_strang_grad", "oracle_loss"):
        getattr(lib, name).restype = c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _configure(ctypes.CDLL(_LIB_PATH))
    return _lib


def use_library(path: str) -> None:
    """Route every oracle call of this process through the compiled oracle at `path` (a build
    of a modified copy of cme_oracle.c: the test that plants mistakes in the oracle and checks
    that its pins catch them)."""
    global _lib
    with _lock:
        _lib = _configure(ctypes.CDLL(path))


def _modes(inst) -> int:
    """Physical mode count M of an instance (the centred M of its N modes; default N)."""
    M = getattr(inst, "M", None)
    return int(M) if M else int(inst.N)


def _kerr(inst):
    """Per-mode Kerr coefficients g0_mu of an instance (centred, float64), or None: the
    instance's g0 on every mode."""
    g = getattr(inst, "g0_mu", None)
    return None if g is None else np.ascontiguousarray(g, dtype=np.float64)


def _dpo(a):
    """Pointer to a float64 array, or NULL for None."""
    return None if a is None else _dp(a)


def _cbuf(z) -> np.ndarray:
    z = np.ascontiguousarray(np.asarray(z, dtype=np.complex128))
    return np.ascontiguousarray(z.view(np.float64).copy())


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc: int):
    if rc != 0:
        raise ValueError(f"oracle call failed with code {rc}")


def fwm(D, linear: bool = False, M: int | None = None) -> np.ndarray:
    """Direct FWM sum (Eq. 2 / Eq. 3) of a centred complex vector; M = physical modes (the
    centred M of the N; default all), the others treated as padding."""
    d = _cbuf(D)
    N = d.size // 2
    out = np.empty_like(d)
    _check(_load().oracle_fwm(N, int(linear), int(M or N), _dp(d), _dp(out)))
    return out.view(np.complex128)


def rhs(D, g0: float, kappa_ext: float, A_in: complex, linear: bool = False,
        M: int | None = None, g0_mu=None) -> np.ndarray:
    """F(D) = delta_{mu,0} sqrt(kappa_ext) A_in + i g0 FWM(D); with g0_mu (N values, centred)
    the Kerr coefficient of output mode mu is g0_mu[mu] instead of g0."""
    d = _cbuf(D)
    N = d.size // 2
    out = np.empty_like(d)
    g = None if g0_mu is None else np.ascontiguousarray(g0_mu, dtype=np.float64)
    _check(_load().oracle_rhs(N, int(linear), int(M or N), g0, _dpo(g), kappa_ext,
                              complex(A_in).real, complex(A_in).imag, _dp(d), _dp(out)))
    return out.view(np.complex128)


def integrate(inst, h: float, nsteps: int, method: int = RK4IP, linear: bool = False,
              D=None) -> np.ndarray:
    """Advance one instance (workloads.Instance-like) by nsteps of the chosen integrator.
    Returns the final field in the rotating (D) frame, centred order."""
    d = _cbuf(inst.D0 if D is None else D)
    kap = np.ascontiguousarray(inst.kappa, dtype=np.float64)
    om = np.ascontiguousarray(inst.omega, dtype=np.float64)
    A = complex(inst.A_in)
    g = _kerr(inst)
    _check(_load().oracle_integrate(method, inst.N, int(linear), _modes(inst), _dp(kap), _dp(om),
                                    inst.g0, _dpo(g), inst.kappa_ext, A.real, A.imag, inst.sigma,
                                    h, int(nsteps), _dp(d)))
    return d.view(np.complex128)


def integrate_eq1(inst, tau0: float, h: float, nsteps: int, A=None, linear: bool = False):
    """Classic RK4 on Eq. 1 as printed (laboratory frame, explicit phase factors)."""
    a = _cbuf(inst.D0 if A is None else A)
    kap = np.ascontiguousarray(inst.kappa, dtype=np.float64)
    om = np.ascontiguousarray(inst.omega, dtype=np.float64)
    Ain = complex(inst.A_in)
    _check(_load().oracle_integrate_eq1(inst.N, int(linear), _dp(kap), _dp(om), inst.g0,
                                        inst.kappa_ext, Ain.real, Ain.imag, inst.sigma, tau0, h,
                                        int(nsteps), _dp(a)))
    return a.view(np.complex128)


def dft(x, sign: int) -> np.ndarray:
    """Naive transform over the mode number: sign=+1 modes -> time, sign=-1 time -> modes."""
    d = _cbuf(x)
    N = d.size // 2
    out = np.empty_like(d)
    _check(_load().oracle_dft(N, sign, _dp(d), _dp(out)))
    return out.view(np.complex128)


def invariants(D, omega, g0: float, sigma: float, linear: bool = False):
    """(sum |D|^2, H) of the lossless, unpumped system."""
    d = _cbuf(D)
    N = d.size // 2
    om = np.ascontiguousarray(omega, dtype=np.float64)
    out = np.empty(2)
    _check(_load().oracle_invariants(N, int(linear), _dp(om), g0, sigma, _dp(d), _dp(out)))
    return float(out[0]), float(out[1])


def fwm_vjp(D, Wbar, linear: bool = False, M: int | None = None) -> np.ndarray:
    """J^H Wbar of the direct FWM sum at D (cotangent convention dL/dRe + i dL/dIm)."""
    d = _cbuf(D)
    wb = _cbuf(Wbar)
    N = d.size // 2
    out = np.empty_like(d)
    _check(_load().oracle_fwm_vjp(N, int(linear), int(M or N), _dp(d), _dp(wb), _dp(out)))
    return out.view(np.complex128)


def log_spectrum_loss(inst, h: float, nsteps: int, target, eps: float = 1e-20,
                      linear: bool = False, D0=None, method: int = RK4IP) -> float:
    """L = sum_mu (log10(|D_mu|^2 + eps) - T_mu)^2 after nsteps RK4IP (or Strang) steps."""
    d = _cbuf(inst.D0 if D0 is None else D0)
    kap = np.ascontiguousarray(inst.kappa, dtype=np.float64)
    om = np.ascontiguousarray(inst.omega, dtype=np.float64)
    T = np.ascontiguousarray(target, dtype=np.float64)
    A = complex(inst.A_in)
    out = np.zeros(1)
    g = _kerr(inst)
    if method == RK4IP:
        _check(_load().oracle_rk4ip_loss(inst.N, int(linear), _modes(inst), _dp(kap), _dp(om),
                                         inst.g0, _dpo(g), inst.kappa_ext, A.real, A.imag,
                                         inst.sigma, h, int(nsteps), _dp(d), _dp(T), eps,
                                         _dp(out)))
    else:
        if method != STRANG or linear:
            raise ValueError("loss: RK4IP (circular or linear) or Strang (circular)")
        _check(_load().oracle_loss(1, inst.N, _modes(inst), _dp(kap), _dp(om), inst.g0, _dpo(g),
                                   inst.kappa_ext, A.real, A.imag, inst.sigma, h, int(nsteps),
                                   _dp(d), _dp(T), eps, _dp(out)))
    return float(out[0])


def log_spectrum_grad(inst, h: float, nsteps: int, target, eps: float = 1e-20,
                      linear: bool = False, method: int = RK4IP):
    """Discrete adjoint of the RK4IP (or Strang) run for the log-spectrum loss.  Returns a dict
    with the loss and the gradients with respect to the initial field (complex,
    dL/dRe + i dL/dIm), sigma, the omega_mu array, the kappa_mu array, A_in (complex) and, for
    omega_mu = D2 mu^2/2 + D3 mu^3/6, D2 and D3."""
    N = inst.N
    d = _cbuf(inst.D0)
    kap = np.ascontiguousarray(inst.kappa, dtype=np.float64)
    om = np.ascontiguousarray(inst.omega, dtype=np.float64)
    T = np.ascontiguousarray(target, dtype=np.float64)
    A = complex(inst.A_in)
    loss = np.zeros(1)
    gD0 = np.zeros(2 * N)
    gLi = np.zeros(N)
    gLr = np.zeros(N)
    gP = np.zeros(2)
    if method == RK4IP:
        _check(_load().oracle_rk4ip_grad(N, int(linear), _modes(inst), _dp(kap), _dp(om),
                                         inst.g0, _dpo(_kerr(inst)), inst.kappa_ext, A.real,
                                         A.imag, inst.sigma, h,
                                         int(nsteps), _dp(d), _dp(T), eps, _dp(loss), _dp(gD0),
                                         _dp(gLi), _dp(gLr), _dp(gP)))
    else:
        if method != STRANG or linear or _kerr(inst) is not None:
            raise ValueError("gradient: RK4IP (circular or linear), or Strang (circular, "
                             "constant g0)")
        _check(_load().oracle_strang_grad(N, _modes(inst), _dp(kap), _dp(om), inst.g0,
                                          inst.kappa_ext, A.real, A.imag, inst.sigma, h,
                                          int(nsteps), _dp(d), _dp(T), eps, _dp(loss), _dp(gD0),
                                          _dp(gLi), _dp(gLr), _dp(gP)))
    mu = np.arange(N) - N // 2
    # Im L_mu = omega_mu - omega_0 - sigma; Re L_mu = -kappa_mu / 2
    g_omega = gLi.copy()
    g_omega[N // 2] -= gLi.sum()
    return {
        "loss": float(loss[0]),
        "D0": gD0.view(np.complex128),
        "sigma": float(-gLi.sum()),
        "omega": g_omega,
        "kappa": -0.5 * gLr,
        "A_in": complex(gP[0], gP[1]) * np.sqrt(inst.kappa_ext),
        "D2": float(np.sum(g_omega * mu * mu / 2.0)),
        "D3": float(np.sum(g_omega * mu ** 3 / 6.0)),
    }


def to_lab_frame(inst, D, tau: float) -> np.ndarray:
    """A_mu = D_mu exp(-i (omega_mu - omega_0 - sigma) tau)."""
    om = np.asarray(inst.omega, dtype=np.float64)
    ph = (om - om[inst.N // 2] - inst.sigma) * tau
    return np.asarray(D) * np.exp(-1j * ph)


def rel_l2(x, y) -> float:
    """||x - y||_2 / ||y||_2 over all modes."""
    x = np.asarray(x)
    y = np.asarray(y)
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))
