"""Dot-product pins of the oracle's discrete adjoints (RK4IP and Strang, log-power-spectrum
loss).  A tangent-linear model of the same discrete runs -- forward-mode derivatives of each
step, written here from the integrators' definitions (Sec. 2: RK4IP in the interaction
picture, the Strang split step with the exact Kerr phase and the exact affine linear flow),
with the four-wave-mixing sum evaluated through numpy's FFT (Eq. 4) -- gives J v up to
rounding.  The oracle's adjoint gives J^H w for the loss cotangent w of the final field.  So
Re <w, J v> = Re <J^H w, v> must hold to rounding, for directions of the initial field and for
the parameters sigma, A_in, D2, D3 and kappa, with padding modes, the linear (de-aliased) sum
and per-mode Kerr coefficients: a far tighter pin than finite differences.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_1307_3428_gb300 import workloads as wl


def _eq4(x, linear):
    """Circular FWM sum of a centred vector through Eq. 4 (a = unnormalised inverse DFT over
    mu, FWM = DFT(|a|^2 a) / N), or the linear (non-wrapping) sum: the circular sum of the
    vector embedded in 2N slots, whose central N entries no wrapped triple reaches."""
    N = x.size
    if linear:
        z = np.zeros(2 * N, complex)
        z[N // 2:N // 2 + N] = x
        return _eq4(z, False)[N // 2:N // 2 + N]
    a = N * np.fft.ifft(np.fft.ifftshift(x))
    return np.fft.fftshift(np.fft.fft(np.abs(a) ** 2 * a)) / N


def _eq4_jvp(x, dx, linear):
    """Directional derivative of _eq4 at x along dx: d(|a|^2 a) = 2 |a|^2 da + a^2 conj(da)."""
    N = x.size
    if linear:
        z, dz = np.zeros(2 * N, complex), np.zeros(2 * N, complex)
        z[N // 2:N // 2 + N], dz[N // 2:N // 2 + N] = x, dx
        return _eq4_jvp(z, dz, False)[N // 2:N // 2 + N]
    a = N * np.fft.ifft(np.fft.ifftshift(x))
    da = N * np.fft.ifft(np.fft.ifftshift(dx))
    return np.fft.fftshift(np.fft.fft(2 * np.abs(a) ** 2 * da + a * a * np.conj(da))) / N


def mask_of(inst):
    """Physical modes: the centred M of the N (all N without padding)."""
    N = inst.N
    M = getattr(inst, "M", None) or N
    i = np.arange(N)
    return (i >= N // 2 - M // 2) & (i < N // 2 - M // 2 + M)


def fwm(D, m=None, linear=False):
    """FWM sum over the physical modes m, zero on the others."""
    m = np.ones(D.size, bool) if m is None else m
    return np.where(m, _eq4(np.where(m, D, 0), linear), 0)


def fwm_jvp(D, dD, m=None, linear=False):
    m = np.ones(D.size, bool) if m is None else m
    return np.where(m, _eq4_jvp(np.where(m, D, 0), np.where(m, dD, 0), linear), 0)


def operator(inst):
    """L_mu = -kappa_mu / 2 + i (omega_mu - omega_0 - sigma) and the pump vector (mode 0)."""
    N, c = inst.N, inst.N // 2
    L = -0.5 * np.asarray(inst.kappa) + 1j * (np.asarray(inst.omega) - inst.omega[c] - inst.sigma)
    P = np.zeros(N, complex)
    P[c] = np.sqrt(inst.kappa_ext) * inst.A_in
    return L, P


def rk4ip_tangent(inst, h, n, dD0, dL, dP, linear=False):
    """n RK4IP steps (E = exp(L h / 2); k1 = E F(D), k2 = F(E D + h/2 k1), k3 = F(E D + h/2 k2),
    k4 = F(E (E D + h k3)), D' = E (E D + h/6 (k1 + 2 k2 + 2 k3)) + h/6 k4, F = P + i g0 FWM,
    g0 per output mode where the instance has per-mode coefficients; padding modes start at
    zero and receive no FWM term) with the tangent of every quantity along (dD0, dL, dP)."""
    L, P = operator(inst)
    m = mask_of(inst)
    g = inst.g0 if getattr(inst, "g0_mu", None) is None else np.asarray(inst.g0_mu)
    E = np.exp(0.5 * h * L)
    dE = 0.5 * h * dL * E

    def F(x):
        return P + 1j * g * fwm(x, m, linear)

    def dF(x, dx):
        return dP + 1j * g * fwm_jvp(x, dx, m, linear)

    D = np.where(m, np.array(inst.D0, complex), 0)
    dD = np.where(m, np.array(dD0, complex), 0)
    for _ in range(n):
        AI, dAI = E * D, dE * D + E * dD
        f1 = F(D)
        k1, dk1 = E * f1, dE * f1 + E * dF(D, dD)
        x2, dx2 = AI + 0.5 * h * k1, dAI + 0.5 * h * dk1
        k2, dk2 = F(x2), dF(x2, dx2)
        x3, dx3 = AI + 0.5 * h * k2, dAI + 0.5 * h * dk2
        k3, dk3 = F(x3), dF(x3, dx3)
        y, dy = AI + h * k3, dAI + h * dk3
        x4, dx4 = E * y, dE * y + E * dy
        k4, dk4 = F(x4), dF(x4, dx4)
        s = AI + h / 6 * (k1 + 2 * k2 + 2 * k3)
        ds = dAI + h / 6 * (dk1 + 2 * dk2 + 2 * dk3)
        D, dD = E * s + h / 6 * k4, dE * s + E * ds + h / 6 * dk4
    return D, dD


def strang_tangent(inst, h, n, dD0, dL, dP, linear=False):
    """n Strang steps (exact linear+pump flow over h/2, D -> E D + c on mode 0 with
    c = (E_0 - 1) / L_0 P_0; exact Kerr flow a -> a exp(i g0 |a|^2 h) of a = IDFT(D), D = DFT(a)/N;
    the linear flow again; padding modes start at zero and the Kerr flow leaves them there)
    with the tangent of every quantity along (dD0, dL, dP)."""
    assert not linear
    L, P = operator(inst)
    m = mask_of(inst)
    N, c, g0 = inst.N, inst.N // 2, inst.g0
    E = np.exp(0.5 * h * L)
    dE = 0.5 * h * dL * E
    L0, E0 = L[c], E[c]
    c0 = (E0 - 1.0) / L0 * P[c]
    dc0 = ((0.5 * h * dL[c] * E0) / L0 - (E0 - 1.0) * dL[c] / L0 ** 2) * P[c] + (E0 - 1.0) / L0 * dP[c]

    def half_flow(D, dD):
        D1, dD1 = E * D, dE * D + E * dD
        D1[c] += c0
        dD1[c] += dc0
        return D1, dD1

    def kerr(D, dD):
        a = N * np.fft.ifft(np.fft.ifftshift(D))
        da = N * np.fft.ifft(np.fft.ifftshift(dD))
        u = np.exp(1j * g0 * h * np.abs(a) ** 2)
        dph = g0 * h * 2.0 * np.real(np.conj(a) * da)
        b, db = a * u, u * (da + 1j * a * dph)
        return (np.where(m, np.fft.fftshift(np.fft.fft(b)) / N, 0),
                np.where(m, np.fft.fftshift(np.fft.fft(db)) / N, 0))

    D = np.where(m, np.array(inst.D0, complex), 0)
    dD = np.where(m, np.array(dD0, complex), 0)
    for _ in range(n):
        D, dD = half_flow(D, dD)
        D, dD = kerr(D, dD)
        D, dD = half_flow(D, dD)
    return D, dD


def loss_cotangent(D, T, eps):
    """w = dL/dRe D + i dL/dIm D of L = sum (log10(|D|^2 + eps) - T)^2."""
    p = np.abs(D) ** 2 + eps
    return 4.0 * (np.log10(p) - T) * D / (p * np.log(10.0))


def _instance(N, seed):
    inst = wl.make_instance(N, 0.05, 0.01, 1.3, 1.4 + 0.2j, 0.05, seed=seed)
    rng = np.random.default_rng(seed + 1)
    inst.kappa = rng.uniform(0.8, 1.2, N)   # per-mode losses: the kappa direction is not flat
    return inst


def _target(N, seed):
    rng = np.random.default_rng(seed)
    return np.log10(rng.uniform(1e-4, 0.5, N))


METHODS = {oracle.RK4IP: rk4ip_tangent, oracle.STRANG: strang_tangent}

# (integrator, N, physical modes M, linear sum, per-mode Kerr coefficients)
CASES = [
    (oracle.RK4IP, 8, None, False, False),
    (oracle.RK4IP, 16, None, False, False),
    (oracle.RK4IP, 16, 13, False, False),
    (oracle.RK4IP, 8, None, True, False),
    (oracle.RK4IP, 16, None, False, True),
    (oracle.RK4IP, 16, 11, True, True),
    (oracle.STRANG, 8, None, False, False),
    (oracle.STRANG, 16, None, False, False),
    (oracle.STRANG, 16, 13, False, False),
]


def _case(N, M, kerr, seed):
    inst = _instance(N, seed)
    if M:
        inst.M = M
    if kerr:
        inst.g0_mu = np.random.default_rng(seed + 2).uniform(0.5, 1.5, N)
    return inst


@pytest.mark.parametrize("method,N,M,linear,kerr", CASES)
def test_tangent_model_forward_matches_the_oracle(method, N, M, linear, kerr):
    """The model's own forward run is the oracle's (its FWM is the direct sum's: Eq. 4 = Eq. 3,
    over the physical modes, circular or linear)."""
    inst = _case(N, M, kerr, 3 + N)
    D = np.random.default_rng(4).standard_normal(N) * (1 + 1j)
    m = mask_of(inst)
    ref = oracle.fwm(D, linear, M)
    assert np.max(np.abs(fwm(D, m, linear) - ref)) <= 1e-12 * np.max(np.abs(ref))
    z = np.zeros(N, complex)
    got, _ = METHODS[method](inst, 0.02, 30, z, z, z, linear)
    assert oracle.rel_l2(got, oracle.integrate(inst, 0.02, 30, method, linear)) <= 1e-12


@pytest.mark.parametrize("method,N,M,linear,kerr", CASES)
def test_adjoint_dot_product(method, N, M, linear, kerr):
    h, n, eps = 0.02, 40, 1e-20
    inst = _case(N, M, kerr, 20 + N)
    T = _target(N, 30 + N)
    g = oracle.log_spectrum_grad(inst, h, n, T, eps=eps, linear=linear, method=method)
    run = METHODS[method]
    z = np.zeros(N, complex)
    Dn, _ = run(inst, h, n, z, z, z, linear)
    w = loss_cotangent(Dn, T, eps)
    mu = (np.arange(N) - N // 2).astype(float)
    c = N // 2
    e0 = np.zeros(N, complex)
    e0[c] = np.sqrt(inst.kappa_ext)

    def directional(dD0=z, dL=z, dP=z):
        _, dDn = run(inst, h, n, dD0, dL, dP, linear)
        return float(np.real(np.vdot(w, dDn)))

    scale = np.max(np.abs(g["D0"]))
    checks = [
        ("sigma", directional(dL=-1j * np.ones(N)), g["sigma"]),
        ("D2", directional(dL=1j * mu ** 2 / 2), g["D2"]),
        ("D3", directional(dL=1j * mu ** 3 / 6), g["D3"]),
        ("kappa", directional(dL=-0.5 * np.ones(N) + 0j), float(np.sum(g["kappa"]))),
        ("A_re", directional(dP=e0), g["A_in"].real),
        ("A_im", directional(dP=1j * e0), g["A_in"].imag),
    ]
    for name, jvp, vjp in checks:
        assert abs(jvp - vjp) <= 1e-11 * max(abs(jvp), abs(g["loss"])), (name, jvp, vjp)
    rng = np.random.default_rng(40 + N)
    for _ in range(4):
        v = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        jvp = directional(dD0=v)
        vjp = float(np.real(np.vdot(g["D0"], v)))
        assert abs(jvp - vjp) <= 1e-11 * max(abs(jvp), scale * np.linalg.norm(v)), (jvp, vjp)
