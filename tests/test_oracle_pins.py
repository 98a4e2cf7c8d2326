"""Pins of the FP64 oracle against results fixed by the paper's equations and by mathematics:
brute-force enumeration of the FWM constraint, library transforms, closed-form stationary
states, exact special cases, conservation laws, convergence orders, the change of frame from
Eq. 1 as printed, and modulational-instability growth rates.  CPU only."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import closed_forms as cf
from oracle import fft_engine
from paper_1307_3428_gb300 import workloads as wl


def rand_field(N, seed, amp=0.5):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(N) + 1j * rng.standard_normal(N)) * amp


def brute_force_fwm(D, linear):
    """Enumerate every (alpha, beta, gamma) of the mode set and keep the triples whose
    alpha - beta + gamma equals mu (modulo N for the circular sum)."""
    N = len(D)
    modes = list(range(-(N // 2), N - N // 2))
    out = np.zeros(N, dtype=complex)
    for mu in modes:
        for a, b, g in itertools.product(modes, repeat=3):
            s = a - b + g
            hit = (s == mu) if linear else ((s - mu) % N == 0)
            if hit:
                out[mu + N // 2] += D[a + N // 2] * np.conj(D[b + N // 2]) * D[g + N // 2]
    return out


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 8])
@pytest.mark.parametrize("linear", [False, True])
def test_fwm_direct_equals_enumeration(N, linear):
    D = rand_field(N, 10 + N)
    got = oracle.fwm(D, linear)
    ref = brute_force_fwm(D, linear)
    assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("N", [2, 4, 8, 16, 32, 64])
@pytest.mark.parametrize("linear", [False, True])
def test_fwm_direct_equals_eq4_fft(N, linear):
    """Eq. 4: the triple sum equals the transform form (numpy.fft as the library routine)."""
    D = rand_field(N, 100 + N)
    got = oracle.fwm(D, linear)
    ref = fft_engine.fwm(D[None, :], linear)[0]
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("N", [1, 2, 3, 8, 16])
def test_naive_transform_matches_numpy(N):
    x = rand_field(N, 7 * N)
    # modes -> time: a_j = sum_mu D_mu e^{+2 pi i j mu/N}
    a = oracle.dft(x, +1)
    ref = np.fft.ifft(np.fft.ifftshift(x)) * N
    assert np.allclose(a, ref, rtol=0, atol=1e-12 * max(1, np.abs(ref).max()))
    # time -> modes (centred output)
    b = oracle.dft(x, -1)
    refb = np.fft.fftshift(np.fft.fft(x))
    assert np.allclose(b, refb, rtol=0, atol=1e-12 * max(1, np.abs(refb).max()))


def test_cw_state_is_fixed_point():
    """The closed-form CW state of every branch makes the full right-hand side vanish."""
    N = 16
    for sigma, Ain in [(2.5, 2.0), (4.0, 2.5), (-1.0, 2.5), (0.5, 1.0)]:
        for P in cf.cw_powers(sigma, Ain, 1.0, 0.5, 1.0):
            D = np.zeros(N, dtype=complex)
            D[N // 2] = cf.cw_field(P, sigma, Ain, 1.0, 0.5, 1.0)
            F = oracle.rhs(D, 1.0, 0.5, Ain)
            L0 = -0.5 + 1j * (0.0 - sigma)
            res = F.copy()
            res[N // 2] += L0 * D[N // 2]
            assert np.max(np.abs(res)) < 1e-13


def test_cw_roots_of_config_one():
    """sigma=2.5, kappa_ext |A_in|^2 = 2: three stationary powers, lower branch ~0.449."""
    Ps = cf.cw_powers(2.5, 2.0, 1.0, 0.5, 1.0)
    assert len(Ps) == 3
    assert abs(Ps[0] - 0.449) < 1e-3 and abs(Ps[1] - 1.42) < 1e-2 and abs(Ps[2] - 3.12) < 1e-2
    # the generator's initial field sits on the lower branch
    inst = wl.plain64()
    assert abs(abs(inst.instances[0].D0[32]) ** 2 - Ps[0]) < 1e-3


def test_single_mode_closed_form():
    """kappa=0, no pump, only mu=0 excited: an exact phase rotation."""
    N = 8
    inst = wl.random_instance(N, 3, kappa=0.0, A_in=0.0, sigma=0.7, D2=0.03)
    D0 = np.zeros(N, dtype=complex)
    D0[N // 2] = 0.9 + 0.4j
    tau, h = 1.0, 0.01
    exact = cf.single_mode(D0[N // 2], inst.sigma, inst.g0, tau)
    Ds = oracle.integrate(inst, h, 100, oracle.STRANG, D=D0)
    assert abs(Ds[N // 2] - exact) < 1e-13
    assert np.max(np.abs(np.delete(Ds, N // 2))) < 1e-13   # transform round-off only
    errs = []
    for n in (100, 200):
        Dr = oracle.integrate(inst, tau / n, n, oracle.RK4IP, D=D0)
        errs.append(abs(Dr[N // 2] - exact))
    assert errs[0] < 1e-8
    assert 12 < errs[0] / errs[1] < 20   # fourth order


def test_linear_affine_exact():
    """g0 = 0: Strang's linear substeps are the exact affine flow; with no pump RK4IP is the
    exact exponential."""
    N = 16
    inst = wl.random_instance(N, 5, g0=0.0, A_in=1.3 - 0.4j, sigma=1.7, D2=0.05)
    L = -0.5 * inst.kappa + 1j * (inst.omega - inst.omega[N // 2] - inst.sigma)
    pump = np.sqrt(inst.kappa_ext) * inst.A_in
    tau, n = 0.8, 40
    exact = cf.linear_affine(inst.D0, L, pump, tau)
    Ds = oracle.integrate(inst, tau / n, n, oracle.STRANG)
    assert np.max(np.abs(Ds - exact)) < 1e-13
    inst0 = wl.random_instance(N, 5, g0=0.0, A_in=0.0, sigma=1.7, D2=0.05)
    exact0 = np.exp(L * tau) * inst0.D0
    Dr = oracle.integrate(inst0, tau / n, n, oracle.RK4IP)
    assert np.max(np.abs(Dr - exact0)) < 1e-14


@pytest.mark.parametrize("linear", [False, True])
def test_lossless_invariants(linear):
    """kappa=0, no pump: sum|D|^2 and H are invariants; RK4IP drift falls as h^4."""
    N = 16
    inst = wl.random_instance(N, 11, kappa=0.0, A_in=0.0, sigma=0.4, D2=0.1, amp=0.3)
    n0, h0 = oracle.invariants(inst.D0, inst.omega, inst.g0, inst.sigma, linear)
    drifts = []
    for n in (100, 200):
        D = oracle.integrate(inst, 2.0 / n, n, oracle.RK4IP, linear=linear)
        n1, h1 = oracle.invariants(D, inst.omega, inst.g0, inst.sigma, linear)
        drifts.append(abs(h1 - h0) + abs(n1 - n0))
    assert drifts[0] < 1e-6 * n0
    assert 12 < drifts[0] / drifts[1] < 20   # h^4
    if not linear:
        D = oracle.integrate(inst, 0.02, 100, oracle.STRANG)
        n1, _ = oracle.invariants(D, inst.omega, inst.g0, inst.sigma)
        assert abs(n1 - n0) < 1e-12 * n0


def test_convergence_orders():
    """RK4IP and plain RK4 are fourth order, Strang second order (Richardson ratios)."""
    N = 16
    inst = wl.random_instance(N, 21, amp=0.4, sigma=1.5, A_in=1.2, D2=0.05)
    tau = 1.0
    ref = oracle.integrate(inst, tau / 1600, 1600, oracle.RK4IP)
    for method, order in ((oracle.RK4IP, 4), (oracle.RK4, 4), (oracle.STRANG, 2)):
        e = [oracle.rel_l2(oracle.integrate(inst, tau / n, n, method), ref) for n in (50, 100)]
        ratio = e[0] / e[1]
        assert 0.75 * 2 ** order < ratio < 1.3 * 2 ** order, (method, e, ratio)


def test_frame_change_from_eq1():
    """Eq. 1 as printed (lab frame, explicit phases, pump e^{i sigma tau}) integrated with RK4
    agrees with the rotating-frame RK4IP after A = D exp(-i(omega_mu - omega_0 - sigma) tau).
    A constant offset in omega_mu leaves both unchanged."""
    N = 8
    inst = wl.random_instance(N, 31, amp=0.5, sigma=1.1, A_in=0.9 + 0.3j, D2=0.2)
    inst.omega = inst.omega + 0.05 * (np.arange(N) - N // 2) ** 3 / 6.0
    tau, n = 0.5, 500
    A_lab = oracle.integrate_eq1(inst, 0.0, tau / n, n)
    D = oracle.integrate(inst, tau / n, n, oracle.RK4IP)
    assert oracle.rel_l2(oracle.to_lab_frame(inst, D, tau), A_lab) < 1e-9
    inst.omega = inst.omega + 3.0
    A_lab2 = oracle.integrate_eq1(inst, 0.0, tau / n, n)
    D2 = oracle.integrate(inst, tau / n, n, oracle.RK4IP)
    assert oracle.rel_l2(A_lab2, A_lab) < 1e-9
    assert oracle.rel_l2(D2, D) < 1e-13


def test_mi_growth_rate():
    """A seeded sideband pair on the CW grows at the closed-form MI rate."""
    N, D2, sigma, Ain = 32, -0.1, 0.0, np.sqrt(2.5)
    P = cf.cw_powers(sigma, Ain, 1.0, 0.5, 1.0)
    assert len(P) == 1 and abs(P[0] - 1.0) < 1e-12
    inst = wl.make_instance(N, D2, 0.0, sigma, Ain, 0.0, seed=0)
    m = 6
    D0 = inst.D0.copy()
    D0[N // 2 + m] += 1e-7
    D0[N // 2 - m] += 1e-7j
    lam = cf.mi_rates(P[0], lambda k: D2 * k * k / 2, sigma, 1.0, 1.0)(m).real
    h = 0.01
    Da = oracle.integrate(inst, h, 500, oracle.RK4IP, D=D0)
    Db = oracle.integrate(inst, h, 500, oracle.RK4IP, D=Da)
    amp = lambda D: np.hypot(abs(D[N // 2 + m]), abs(D[N // 2 - m]))
    rate = np.log(amp(Db) / amp(Da)) / 5.0
    assert abs(rate - lam) < 1e-3 * lam
    assert amp(Db) < 1e-3   # still linear regime


def test_driven_steady_state_lower_branch():
    """Started from the vacuum, the damped-driven system settles on the lower CW branch."""
    N = 16
    inst = wl.make_instance(N, 0.04, 0.0, 2.5, 2.0, 1e-6, seed=4, cw=False)
    P = cf.cw_powers(2.5, 2.0, 1.0, 0.5, 1.0)[0]
    dev = []
    for h in (0.04, 0.02):
        D = oracle.integrate(inst, h, int(round(100.0 / h)), oracle.RK4IP)
        dev.append(abs(abs(D[N // 2]) ** 2 - P))
        assert np.max(np.abs(np.delete(D, N // 2))) < 1e-12
    # the fixed point of the discrete map sits O(h^4) away from the exact one
    assert dev[0] < 1e-6 and 12 < dev[0] / dev[1] < 20


@pytest.mark.parametrize("method", ["rk4ip", "strang", "rk4ip_linear"])
def test_fft_engine_matches_direct(method):
    N = 16
    insts = [wl.random_instance(N, 40 + k, amp=0.5, sigma=0.5 * k, A_in=1.0 + 0.5j * k,
                                D2=0.04) for k in range(3)]
    batch = fft_engine.Batch(insts)
    h, n = 0.01, 60
    if method == "rk4ip":
        got = fft_engine.rk4ip(batch, h, n)
        ref = [oracle.integrate(i, h, n, oracle.RK4IP) for i in insts]
    elif method == "strang":
        got = fft_engine.strang(batch, h, n)
        ref = [oracle.integrate(i, h, n, oracle.STRANG) for i in insts]
    else:
        got = fft_engine.rk4ip(batch, h, n, linear=True)
        ref = [oracle.integrate(i, h, n, oracle.RK4IP, linear=True) for i in insts]
    for g, r in zip(got, ref):
        assert oracle.rel_l2(g, r) < 1e-13
