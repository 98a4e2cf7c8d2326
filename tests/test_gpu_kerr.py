"""Per-mode Kerr coefficients g0_mu (cme_set_kerr): the output mode's four-wave-mixing term
carries g0_mu, applied as a per-mode factor after the forward transform of Eq. 4.  Against the
oracle (direct sum for the right-hand side and short runs, the Eq. 4 engine for longer ones) on
every launch path: one block per instance, thread-block clusters, the persistent work-list
kernel, the four-step large-N kernels, and the discrete adjoint."""
import numpy as np
import pytest

import oracle
from oracle import fft_engine
from paper_1307_3428_gb300 import cme
from paper_1307_3428_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {cme.FP64: 1e-10, cme.FP32: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()
    cme.load()


def rel(x, y):
    return float(np.linalg.norm(np.asarray(x) - np.asarray(y)) / np.linalg.norm(np.asarray(y)))


def kerr_set(N, seed, count, slope=0.4):
    """`count` random instances, every other one with a frequency-dependent Kerr slope (the
    others keep their scalar g0, in the same launch group)."""
    amp = 0.3 * min(1.0, np.sqrt(64.0 / N))
    insts = []
    for k in range(count):
        i = wl.random_instance(N, seed + k, amp=amp, sigma=0.5 * k, A_in=1.0 + 0.2j * k,
                               g0=0.8 + 0.2 * k)
        if k % 2 == 0:
            i.g0_mu = wl.kerr_slope(i.g0, N, slope * (1 + k))
        insts.append(i)
    return insts


def batch_of(insts, prec, **kw):
    return cme.Batch([cme.Instance.from_workload(i) for i in insts], precision=prec, **kw)


@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
@pytest.mark.parametrize("N", [4, 16, 64, 256])
def test_rhs_matches_direct_sum(N, prec):
    insts = kerr_set(N, 1100, 3)
    got = batch_of(insts, prec).split(batch_of(insts, prec).eval_rhs())
    for g, inst in zip(got, insts):
        ref = oracle.rhs(inst.D0, inst.g0, inst.kappa_ext, inst.A_in, g0_mu=inst.g0_mu)
        tol = 1e-12 if prec == cme.FP64 else 3e-6
        assert np.max(np.abs(g - ref)) <= tol * np.max(np.abs(ref)) * max(1, np.log2(N))


@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
def test_rk4ip_one_block_against_direct_sum(prec):
    insts = kerr_set(64, 1200, 4)
    b = batch_of(insts, prec)
    b.step(1e-3, 50)
    for g, inst in zip(b.split(b.get_state()), insts):
        assert rel(g, oracle.integrate(inst, 1e-3, 50, oracle.RK4IP)) <= TOL[prec]


@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
@pytest.mark.parametrize("N,kw", [(512, {}), (2048, {"cluster": 4}), (4096, {"cluster": 8}),
                                  (4096, {"radix": 16, "cluster": 1})])
def test_rk4ip_against_eq4_engine(N, kw, prec):
    insts = kerr_set(N, 1300 + N, 3)
    b = batch_of(insts, prec, **kw)
    b.step(1e-3, 30)
    refs = fft_engine.rk4ip(fft_engine.Batch(insts), 1e-3, 30)
    for g, r in zip(b.split(b.get_state()), refs):
        assert rel(g, r) <= TOL[prec]


@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
def test_work_list_kernel_and_large_n(prec):
    """Mixed N in one persistent work-list launch, and N = 8192 on the four-step kernels."""
    insts = kerr_set(64, 1400, 2) + kerr_set(256, 1410, 2) + kerr_set(1024, 1420, 2)
    b = batch_of(insts, prec, persistent=2, use_graph=True)
    b.step(1e-3, 20)
    got = b.split(b.get_state())
    for N in (64, 256, 1024):
        sel = [k for k, i in enumerate(insts) if i.N == N]
        refs = fft_engine.rk4ip(fft_engine.Batch([insts[k] for k in sel]), 1e-3, 20)
        for k, r in zip(sel, refs):
            assert rel(got[k], r) <= TOL[prec], (N, k)
    big = kerr_set(8192, 1430, 2)
    b = batch_of(big, prec)
    b.step(1e-3, 12)
    refs = fft_engine.rk4ip(fft_engine.Batch(big), 1e-3, 12)
    for g, r in zip(b.split(b.get_state()), refs):
        assert rel(g, r) <= TOL[prec]


def test_constant_per_mode_coefficients_equal_scalar_g0():
    insts = [wl.random_instance(256, 1500 + k, amp=0.1, g0=1.3) for k in range(2)]
    ref = batch_of(insts, cme.FP64)
    ref.step(1e-3, 40)
    for i in insts:
        i.g0_mu = np.full(256, 1.3)
    b = batch_of(insts, cme.FP64)
    b.step(1e-3, 40)
    assert rel(b.get_state(), ref.get_state()) <= 1e-14


def test_adjoint_matches_oracle_adjoint():
    h, n = 0.02, 25
    for N in (16, 64):
        insts = []
        for k in range(3):
            i = wl.make_instance(N, 0.05, 0.01, 1.3, 1.4 + 0.2j, 0.05, seed=1600 + k)
            if k != 1:
                i.g0_mu = wl.kerr_slope(1.0, N, 0.3 + 0.2 * k)
            insts.append(i)
        T = [np.log10(np.random.default_rng(1610 + k).uniform(1e-4, 0.5, N)) for k in range(3)]
        g = batch_of(insts, cme.FP64).grad(h, n, np.concatenate(T))
        for k, (inst, t) in enumerate(zip(insts, T)):
            o = oracle.log_spectrum_grad(inst, h, n, t)
            sl = slice(k * N, (k + 1) * N)
            assert abs(g["loss"][k] - o["loss"]) <= 1e-11 * abs(o["loss"])
            for key, ref in (("d_sigma", o["sigma"]), ("d_D2", o["D2"])):
                assert abs(g[key][k] - ref) <= 1e-9 * max(abs(ref), 1e-6 * abs(o["loss"])), key
            assert abs(g["d_A_in"][k] - o["A_in"]) <= 1e-9 * abs(o["A_in"])
            assert np.max(np.abs(g["d_D0"][sl] - o["D0"])) <= 1e-9 * np.max(np.abs(o["D0"]))


def test_strang_batch_refuses_per_mode_coefficients():
    insts = kerr_set(64, 1700, 2)
    with pytest.raises(cme.CmeError) as e:
        batch_of(insts, cme.FP64, integrator=cme.STRANG)
    assert e.value.code == -1


def test_cluster_adjoint_agrees_with_one_block():
    """N = 2048 with per-mode coefficients on 4-block clusters against one block per instance,
    FP64 gradients (the oracle's direct-sum adjoint is out of reach at this size): to 1e-9."""
    N = 2048
    insts = kerr_set(N, 1800, 2)
    T = np.concatenate([np.log10(np.random.default_rng(1810 + k).uniform(1e-4, 0.5, N))
                        for k in range(2)])
    g = {}
    for c in (1, 4):
        b = batch_of(insts, cme.FP64, radix=8, cluster=c)
        g[c] = b.grad(1e-3, 24, T, segment=5)
        b.close()
    for key in g[1]:
        a, r = np.asarray(g[4][key]), np.asarray(g[1][key])
        assert np.linalg.norm(a - r) <= 1e-9 * np.linalg.norm(r), key
