"""Dot-product pins of the oracle's discrete adjoints (RK4IP and Strang, log-power-spectrum
loss).  A tangent-linear model of the same discrete runs -- forward-mode derivatives of each
step, written here from the integrators' definitions (Sec. 2: RK4IP in the interaction
picture, the Strang split step with the exact Kerr phase and the exact affine linear flow),
with the four-wave-mixing sum evaluated through numpy's FFT (Eq. 4) -- gives J v up to
rounding.  The oracle's adjoint gives J^H w for the loss cotangent w of the final field.  So
Re <w, J v> = Re <J^H w, v> must hold to rounding, for directions of the initial field and for
the parameters sigma, A_in, D2, D3 and kappa: a far tighter pin than finite differences.
CPU only."""
import numpy as np
import pytest

import oracle
from paper_1307_3428_gb300 import workloads as wl


def fwm(D):
    """Eq. 4 in centred order: a = unnormalised inverse DFT over mu, FWM = DFT(|a|^2 a) / N."""
    N = D.size
    a = N * np.fft.ifft(np.fft.ifftshift(D))
    return np.fft.fftshift(np.fft.fft(np.abs(a) ** 2 * a)) / N


def fwm_jvp(D, dD):
    """Directional derivative of fwm at D along dD: d(|a|^2 a) = 2 |a|^2 da + a^2 conj(da)."""
    N = D.size
    a = N * np.fft.ifft(np.fft.ifftshift(D))
    da = N * np.fft.ifft(np.fft.ifftshift(dD))
    return np.fft.fftshift(np.fft.fft(2 * np.abs(a) ** 2 * da + a * a * np.conj(da))) / N


def operator(inst):
    """L_mu = -kappa_mu / 2 + i (omega_mu - omega_0 - sigma) and the pump vector (mode 0)."""
    N, c = inst.N, inst.N // 2
    L = -0.5 * np.asarray(inst.kappa) + 1j * (np.asarray(inst.omega) - inst.omega[c] - inst.sigma)
    P = np.zeros(N, complex)
    P[c] = np.sqrt(inst.kappa_ext) * inst.A_in
    return L, P


def rk4ip_tangent(inst, h, n, dD0, dL, dP):
    """n RK4IP steps (E = exp(L h / 2); k1 = E F(D), k2 = F(E D + h/2 k1), k3 = F(E D + h/2 k2),
    k4 = F(E (E D + h k3)), D' = E (E D + h/6 (k1 + 2 k2 + 2 k3)) + h/6 k4, F = P + i g0 FWM)
    with the tangent of every quantity along (dD0, dL, dP)."""
    L, P = operator(inst)
    g0 = inst.g0
    E = np.exp(0.5 * h * L)
    dE = 0.5 * h * dL * E

    def F(x):
        return P + 1j * g0 * fwm(x)

    def dF(x, dx):
        return dP + 1j * g0 * fwm_jvp(x, dx)

    D = np.array(inst.D0, complex)
    dD = np.array(dD0, complex)
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


def strang_tangent(inst, h, n, dD0, dL, dP):
    """n Strang steps (exact linear+pump flow over h/2, D -> E D + c on mode 0 with
    c = (E_0 - 1) / L_0 P_0; exact Kerr flow a -> a exp(i g0 |a|^2 h) of a = IDFT(D), D = DFT(a)/N;
    the linear flow again) with the tangent of every quantity along (dD0, dL, dP)."""
    L, P = operator(inst)
    N, c, g0 = inst.N, inst.N // 2, inst.g0
    E = np.exp(0.5 * h * L)
    dE = 0.5 * h * dL * E
    L0, E0 = L[c], E[c]
    c0 = (E0 - 1.0) / L0 * P[c]
    dc0 = ((0.5 * h * dL[c] * E0) / L0 - (E0 - 1.0) * dL[c] / L0 ** 2) * P[c] + (E0 - 1.0) / L0 * dP[c]

    def linear(D, dD):
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
        return (np.fft.fftshift(np.fft.fft(b)) / N, np.fft.fftshift(np.fft.fft(db)) / N)

    D = np.array(inst.D0, complex)
    dD = np.array(dD0, complex)
    for _ in range(n):
        D, dD = linear(D, dD)
        D, dD = kerr(D, dD)
        D, dD = linear(D, dD)
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


def test_tangent_model_forward_matches_the_oracle():
    """The model's own forward run is the oracle's (its FWM is the direct sum's, Eq. 4 = Eq. 3)."""
    inst = _instance(16, 3)
    D = np.random.default_rng(4).standard_normal(16) * (1 + 1j)
    assert np.max(np.abs(fwm(D) - oracle.fwm(D))) <= 1e-12 * np.max(np.abs(oracle.fwm(D)))
    z = np.zeros(16, complex)
    for method, run in METHODS.items():
        got, _ = run(inst, 0.02, 30, z, z, z)
        ref = oracle.integrate(inst, 0.02, 30, method)
        assert oracle.rel_l2(got, ref) <= 1e-12, method


@pytest.mark.parametrize("method", [oracle.RK4IP, oracle.STRANG])
@pytest.mark.parametrize("N", [8, 16])
def test_adjoint_dot_product(method, N):
    h, n, eps = 0.02, 40, 1e-20
    inst = _instance(N, 20 + N)
    T = _target(N, 30 + N)
    g = oracle.log_spectrum_grad(inst, h, n, T, eps=eps, method=method)
    run = METHODS[method]
    z = np.zeros(N, complex)
    Dn, _ = run(inst, h, n, z, z, z)
    w = loss_cotangent(Dn, T, eps)
    mu = (np.arange(N) - N // 2).astype(float)
    c = N // 2
    e0 = np.zeros(N, complex)
    e0[c] = np.sqrt(inst.kappa_ext)

    def directional(dD0=z, dL=z, dP=z):
        _, dDn = run(inst, h, n, dD0, dL, dP)
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
