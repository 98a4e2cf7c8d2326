"""Physical-mode count M (cme_set_modes; the zero padding of Sec. 2) on the GPU against the
oracle: of N modes only the centred M are physical, the others stay at zero and get no FWM
term.  Covers the paper's case (201 modes in a 256-point transform, where some triples still
wrap around), full de-aliasing (N >= 2M equals the linear sum of the M-mode system), several M
in one launch group, every launch path (per-group, work-list, cluster, four-step) and the
adjoint."""
import copy

import numpy as np
import pytest

import oracle
from oracle import fft_engine
from paper_1307_3428_gb300 import cme
from paper_1307_3428_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()
    cme.load()


def rel(x, y):
    return float(np.linalg.norm(np.asarray(x) - np.asarray(y)) / np.linalg.norm(np.asarray(y)))


def band(N, M):
    first = N // 2 - M // 2
    return np.arange(first, first + M)


def padded(N, M, seed, amp=None, sigma=0.6, A_in=1.2 + 0.2j):
    """A random instance with M physical modes; the padding entries of the initial field hold
    junk, which the library must discard."""
    amp = amp if amp is not None else 0.3 * min(1.0, np.sqrt(64.0 / M))
    inst = wl.random_instance(N, seed, amp=amp, sigma=sigma, A_in=A_in)
    rng = np.random.default_rng(seed + 7)
    junk = (rng.standard_normal(N) + 1j * rng.standard_normal(N)) * 3.0
    keep = np.zeros(N, dtype=bool)
    keep[band(N, M)] = True
    inst.D0 = np.where(keep, inst.D0, junk)
    inst.M = M
    return inst


def zeroed(inst):
    out = inst.D0.copy()
    mask = np.ones(inst.N, dtype=bool)
    mask[band(inst.N, inst.M)] = False
    out[mask] = 0
    return out


def batch_of(insts, prec, integ=cme.RK4IP, **kw):
    return cme.Batch([cme.Instance.from_workload(i) for i in insts], precision=prec,
                     integrator=integ, **kw)


@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
@pytest.mark.parametrize("N,M", [(8, 5), (16, 11), (64, 33), (256, 201)])
def test_padded_rhs_matches_direct_sum(N, M, prec):
    insts = [padded(N, M, 4000 + k) for k in range(2)]
    b = batch_of(insts, prec)
    got = b.split(b.eval_rhs())
    for g, inst in zip(got, insts):
        ref = oracle.rhs(zeroed(inst), inst.g0, inst.kappa_ext, inst.A_in, M=M)
        tol = 1e-12 if prec == cme.FP64 else 3e-6
        assert np.max(np.abs(g - ref)) <= tol * np.max(np.abs(ref)) * max(1, np.log2(N))


@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
@pytest.mark.parametrize("N,M", [(16, 7), (16, 11)])
def test_padded_rk4ip_matches_direct_oracle(N, M, prec):
    insts = [padded(N, M, 4100 + k) for k in range(3)]
    b = batch_of(insts, prec)
    b.step(2e-3, 60)
    got = b.split(b.get_state())
    for g, inst in zip(got, insts):
        ref = oracle.integrate(inst, 2e-3, 60, oracle.RK4IP)
        assert rel(g, ref) <= (1e-12 if prec == cme.FP64 else 1e-5)
        assert np.all(np.delete(g, band(N, M)) == 0)


@pytest.mark.parametrize("integ", [cme.RK4IP, cme.STRANG])
@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
def test_paper_padding_201_in_256(prec, integ):
    """Sec. 2's own case: 201 physical modes zero padded to a 256-point transform."""
    insts = [padded(256, 201, 4200 + k) for k in range(4)]
    b = batch_of(insts, prec, integ)
    b.step(2e-3, 100)
    got = b.split(b.get_state())
    fb = fft_engine.Batch(insts)
    refs = (fft_engine.rk4ip(fb, 2e-3, 100) if integ == cme.RK4IP
            else fft_engine.strang(fb, 2e-3, 100))
    for g, r in zip(got, refs):
        assert rel(g, r) <= (1e-11 if prec == cme.FP64 else 1e-5)
        assert np.all(np.delete(g, band(256, 201)) == 0)


def test_padded_strang_matches_direct_oracle():
    insts = [padded(16, 11, 4250 + k) for k in range(2)]
    b = batch_of(insts, cme.FP64, cme.STRANG)
    b.step(4e-3, 50)
    got = b.split(b.get_state())
    for g, inst in zip(got, insts):
        ref = oracle.integrate(inst, 4e-3, 50, oracle.STRANG)
        assert rel(g, ref) <= 1e-12


@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
def test_padding_to_2m_is_the_dealiased_linear_system(prec):
    """N = 128 holding M = 64 physical modes evolves exactly as the 64-mode system with the
    linear (non-wrapping) four-wave-mixing sum."""
    N, M = 128, 64
    base = wl.random_instance(M, 4300, amp=0.3, sigma=0.4, A_in=1.1)
    inst = copy.deepcopy(base)
    inst.N, inst.M = N, M
    inst.kappa = np.full(N, 1.0)
    inst.kappa[band(N, M)] = base.kappa
    inst.omega = np.zeros(N)
    inst.omega[band(N, M)] = base.omega
    inst.D0 = np.zeros(N, dtype=complex)
    inst.D0[band(N, M)] = base.D0
    b = batch_of([inst], prec)
    b.step(2e-3, 25)
    got = b.get_state()[band(N, M)]
    ref = oracle.integrate(base, 2e-3, 25, oracle.RK4IP, linear=True)
    assert rel(got, ref) <= (1e-12 if prec == cme.FP64 else 1e-5)


@pytest.mark.parametrize("persistent", [1, 2])
def test_several_m_in_one_group_and_mixed_sizes(persistent):
    """Per-instance M inside one launch group (N = 64: M = 64, 40, 33) next to other N, on the
    per-group and the work-list paths."""
    insts = ([padded(64, M, 4400 + M) for M in (64, 40, 33)] +
             [padded(256, 201, 4410), padded(1024, 700, 4411)])
    b = batch_of(insts, cme.FP32, persistent=persistent, use_graph=True)
    b.step(1e-3, 30)
    got = b.split(b.get_state())
    for N in (64, 256, 1024):
        sel = [k for k, i in enumerate(insts) if i.N == N]
        refs = fft_engine.rk4ip(fft_engine.Batch([insts[k] for k in sel]), 1e-3, 30)
        for k, r in zip(sel, refs):
            assert rel(got[k], r) <= 1e-5, (N, k)


@pytest.mark.parametrize("prec,cluster", [(cme.FP64, 0), (cme.FP32, 4)])
def test_padded_cluster_groups(prec, cluster):
    """N = 4096 with M = 3001 on thread-block clusters (FP64 by default, FP32 on request)."""
    insts = [padded(4096, 3001, 4500 + k) for k in range(2)]
    b = batch_of(insts, prec, cluster=cluster)
    b.step(1e-3, 10)
    got = b.split(b.get_state())
    refs = fft_engine.rk4ip(fft_engine.Batch(insts), 1e-3, 10)
    for g, r in zip(got, refs):
        assert rel(g, r) <= (1e-12 if prec == cme.FP64 else 1e-5)


@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
def test_padded_four_step_path(prec):
    """N = 8192 (four-step row/column kernels) with M = 5000."""
    insts = [padded(8192, 5000, 4600 + k) for k in range(2)]
    b = batch_of(insts, prec)
    b.step(2e-4, 40)
    got = b.split(b.get_state())
    refs = fft_engine.rk4ip(fft_engine.Batch(insts), 2e-4, 40)
    for g, r in zip(got, refs):
        assert rel(g, r) <= (1e-12 if prec == cme.FP64 else 1e-5)
        assert np.all(np.delete(g, band(8192, 5000)) == 0)


def target_for(N, seed):
    rng = np.random.default_rng(seed)
    return np.log10(rng.uniform(1e-4, 0.5, N))


@pytest.mark.parametrize("N,M", [(16, 11), (64, 33)])
def test_padded_adjoint_matches_oracle_adjoint(N, M):
    h, n = 0.02, 25
    insts = [padded(N, M, 4700 + k, amp=0.2) for k in range(2)]
    T = [target_for(N, 4710 + k) for k in range(2)]
    b = batch_of(insts, cme.FP64)
    g = b.grad(h, n, np.concatenate(T))
    for k, (inst, t) in enumerate(zip(insts, T)):
        o = oracle.log_spectrum_grad(inst, h, n, t)
        sl = slice(k * N, (k + 1) * N)
        assert abs(g["loss"][k] - o["loss"]) <= 1e-11 * abs(o["loss"])
        assert abs(g["d_sigma"][k] - o["sigma"]) <= 1e-9 * max(abs(o["sigma"]), 1e-6 * abs(o["loss"]))
        assert abs(g["d_A_in"][k] - o["A_in"]) <= 1e-9 * abs(o["A_in"])
        assert np.max(np.abs(g["d_D0"][sl] - o["D0"])) <= 1e-9 * np.max(np.abs(o["D0"]))
        assert np.max(np.abs(g["d_omega"][sl] - o["omega"])) <= 1e-9 * np.max(np.abs(o["omega"]))
