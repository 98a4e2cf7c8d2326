"""Instances spread over a thread-block cluster (cme_options.cluster = C > 1): the C blocks hold
P/C threads each and run a four-step transform, an N/C-point transform inside each block and
C-point transforms in registers, with one all-to-all through distributed shared memory per
transform.

Checked against the oracle (N = 256 with C = 2 against the direct-sum oracle, N = 2048 and
4096 against the oracle's Eq. 4 engine, the adjoint at N = 256 against the oracle's adjoint),
and against the one-block kernels, which round in another order: the two agree to the
precision's rounding."""
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


def batch_of(insts, prec, integ=cme.RK4IP, **kw):
    return cme.Batch([cme.Instance.from_workload(i) for i in insts], precision=prec,
                     integrator=integ, **kw)


def random_set(N, seed, count):
    amp = 0.3 * min(1.0, np.sqrt(64.0 / N))
    return [wl.random_instance(N, seed + k, amp=amp, sigma=0.5 * k, A_in=1.0 + 0.2j * k)
            for k in range(count)]


@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
def test_cluster_n256_rk4ip_matches_direct_sum(prec):
    insts = random_set(256, 3000, 3)
    b = batch_of(insts, prec, cluster=2)
    b.step(1e-3, 6)
    got = b.split(b.get_state())
    for g, inst in zip(got, insts):
        ref = oracle.integrate(inst, 1e-3, 6, oracle.RK4IP)
        assert rel(g, ref) <= (1e-12 if prec == cme.FP64 else 1e-5)


@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
def test_cluster_n256_strang_matches_direct_sum(prec):
    insts = random_set(256, 3100, 3)
    b = batch_of(insts, prec, cme.STRANG, cluster=2)
    b.step(2e-3, 10)
    got = b.split(b.get_state())
    for g, inst in zip(got, insts):
        ref = oracle.integrate(inst, 2e-3, 10, oracle.STRANG)
        assert rel(g, ref) <= (1e-11 if prec == cme.FP64 else 1e-5)


@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
@pytest.mark.parametrize("N,C", [(2048, 2), (2048, 8), (4096, 4), (4096, 8)])
def test_cluster_rk4ip_matches_eq4_engine(N, C, prec):
    insts = random_set(N, 3200 + N, 3)
    b = batch_of(insts, prec, cluster=C)
    b.step(1e-3, 20)
    got = b.split(b.get_state())
    refs = fft_engine.rk4ip(fft_engine.Batch(insts), 1e-3, 20)
    for g, r in zip(got, refs):
        assert rel(g, r) <= (1e-12 if prec == cme.FP64 else 1e-5)


@pytest.mark.parametrize("integ", [cme.RK4IP, cme.STRANG])
@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
@pytest.mark.parametrize("N,C", [(256, 2), (2048, 4), (4096, 2), (4096, 8)])
def test_cluster_agrees_with_one_block(N, C, prec, integ):
    insts = random_set(N, 3300 + N, 3)
    out = {}
    for c in (1, C):
        b = batch_of(insts, prec, integ, radix=8, cluster=c)   # same values per thread
        b.step(1e-3, 37)
        b.synchronize()
        out[c] = b.get_state()
        b.close()
    # measured (GB300): FP64 <= 7.5e-16; FP32 2.1e-7 ... 4.3e-7 (each side 0.9e-7 ... 2.1e-6
    # from FP64, the cluster kernel within 1% of the one-block kernel's own error)
    assert rel(out[C], out[1]) <= (1e-12 if prec == cme.FP64 else 1e-6)


def test_cluster_inside_a_mixed_batch():
    """N = 4096 instances on clusters next to N = 512 and N = 64 groups, one kernel per group on
    concurrent streams, against the Eq. 4 engine."""
    insts = random_set(64, 3400, 2) + random_set(512, 3410, 3) + random_set(4096, 3420, 2)
    b = batch_of(insts, cme.FP32, persistent=1, cluster=4, use_graph=True)
    b.step(1e-3, 10)
    b.step(1e-3, 10)
    got = b.split(b.get_state())
    for N in (64, 512, 4096):
        sel = [k for k, i in enumerate(insts) if i.N == N]
        refs = fft_engine.rk4ip(fft_engine.Batch([insts[k] for k in sel]), 1e-3, 20)
        for k, r in zip(sel, refs):
            assert rel(got[k], r) <= 1e-5, (N, k)


def target_for(N, seed):
    rng = np.random.default_rng(seed)
    return np.log10(rng.uniform(1e-4, 0.5, N))


def test_cluster_adjoint_n256_matches_oracle_adjoint():
    N, h, n = 256, 0.01, 4
    insts = [wl.make_instance(N, 0.05, 0.01, 1.3, 1.4 + 0.2j, 0.05, seed=3500 + k)
             for k in range(2)]
    T = [target_for(N, 3510 + k) for k in range(2)]
    b = batch_of(insts, cme.FP64, cluster=2)
    g = b.grad(h, n, np.concatenate(T))
    for k, (inst, t) in enumerate(zip(insts, T)):
        o = oracle.log_spectrum_grad(inst, h, n, t)
        sl = slice(k * N, (k + 1) * N)
        assert abs(g["loss"][k] - o["loss"]) <= 1e-11 * abs(o["loss"])
        assert abs(g["d_sigma"][k] - o["sigma"]) <= 1e-9 * max(abs(o["sigma"]), 1e-6 * abs(o["loss"]))
        assert abs(g["d_A_in"][k] - o["A_in"]) <= 1e-9 * abs(o["A_in"])
        assert np.max(np.abs(g["d_D0"][sl] - o["D0"])) <= 1e-9 * np.max(np.abs(o["D0"]))
        assert np.max(np.abs(g["d_omega"][sl] - o["omega"])) <= 1e-9 * np.max(np.abs(o["omega"]))


@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
@pytest.mark.parametrize("N,C", [(256, 2), (4096, 8)])
def test_cluster_adjoint_agrees_with_one_block(N, C, prec):
    """Against the one-block FP64 gradient.  In FP64 the cluster gradient agrees with it to
    rounding.  Parameter gradients are sums over modes that cancel, which FP32 determines only
    loosely, so the cluster FP32 gradient must be about as close to FP64 as the one-block FP32
    gradient is: within 4 times its error, or 1e-6.  The two round in different orders, so
    their errors are two draws of the same size: measured on GB300 over the 8 outputs of this
    test and of test_cluster_adjoint_segment_lengths, the ratio of the cluster's error to the
    one-block error lies between 0.75 and 2.51."""
    insts = [wl.make_instance(N, 0.01, 1e-4, 2.0 + k, 2.0, 1e-3, seed=3600 + k) for k in range(2)]
    T = np.concatenate([target_for(N, 3610 + k) for k in range(2)])

    def grad(p, c):
        b = batch_of(insts, p, radix=8, cluster=c)   # same values per thread on both sides
        g = b.grad(2e-4, 40, T, segment=7)
        b.close()
        return g

    ref = grad(cme.FP64, 1)
    got = grad(prec, C)
    if prec == cme.FP64:
        for key in ref:
            assert rel(got[key], ref[key]) <= 1e-9, key
    else:
        one = grad(prec, 1)
        for key in ref:
            e1, eC = rel(one[key], ref[key]), rel(got[key], ref[key])
            assert eC <= max(4 * e1, 1e-6), (key, e1, eC)


@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
def test_plans_run_the_kernels_the_tests_mean(prec):
    """The cluster tests above do run clusters: an explicit cluster request without a radix
    selects the clusters' 8 values per thread, also where the library would otherwise choose 16
    (FP32, N >= 2048).  The library's own choice: 8-block clusters while one block per instance
    would leave SMs idle and the clusters' blocks all stay resident (2 and 64 instances of
    N = 4096), one block per instance for 128 instances."""
    insts = random_set(4096, 3700, 2)
    b = batch_of(insts, prec, cluster=4)
    assert b.plan(0)["radix"] == 8 and b.plan(0)["cluster"] == 4
    b.close()
    for count, cluster in ((2, 8), (64, 8), (128, 1)):
        b = batch_of([insts[k % 2] for k in range(count)], prec)
        p = b.plan(0)
        assert p["cluster"] == cluster, (count, p)
        assert p["radix"] == (16 if cluster == 1 and prec == cme.FP32 else 8), (count, p)
        b.close()


@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
def test_bounded_wait_reports_timeout_and_the_batch_recovers(prec):
    """Failure detection without a device fault: the test switch (cme_debug_fault) makes each
    cluster all-to-all expect one word more than is sent, so its wait runs out of polls.  The
    kernels finish, the instances report status 2, cme_synchronize and cme_grad return
    TIMEOUT, and the same batch then steps correctly again."""
    N = 2048
    insts = random_set(N, 3800, 2)
    b = batch_of(insts, prec, cluster=4)
    D0 = b.get_state()
    b.debug_fault(1)
    b.step(1e-3, 3)
    with pytest.raises(cme.CmeError) as e:
        b.synchronize()
    assert e.value.code == -5
    assert list(b.status()) == [2, 2]
    b.set_state(D0)   # clears the status words
    T = np.concatenate([target_for(N, 3810 + k) for k in range(2)])
    with pytest.raises(cme.CmeError) as e:
        b.grad(1e-3, 4, T)
    assert e.value.code == -5
    b.debug_fault(0)
    b.set_state(D0)
    b.step(1e-3, 10)
    b.synchronize()
    assert list(b.status()) == [0, 0]
    got = b.split(b.get_state())
    refs = fft_engine.rk4ip(fft_engine.Batch(insts), 1e-3, 10)
    for g, r in zip(got, refs):
        assert rel(g, r) <= (1e-12 if prec == cme.FP64 else 1e-5)
    b.close()


@pytest.mark.parametrize("segment", [1, 2, 7])
def test_cluster_adjoint_segment_lengths(segment):
    """The FP32 backward kernel on clusters prefetches the next step's stored data into shared
    memory (two buffers, bulk copies).  Segments of 1, 2 and 7 steps cover the single-step
    segment and both buffer parities; each gradient must be as close to the one-block FP64
    gradient as the one-block FP32 gradient is (within 4 times its error, or 1e-6; see
    test_cluster_adjoint_agrees_with_one_block for the measured spread)."""
    N = 4096
    insts = [wl.make_instance(N, 0.01, 1e-4, 2.0 + k, 2.0, 1e-3, seed=3900 + k) for k in range(2)]
    T = np.concatenate([target_for(N, 3910 + k) for k in range(2)])

    def grad(p, c, seg):
        b = batch_of(insts, p, radix=8, cluster=c)
        g = b.grad(2e-4, 15, T, segment=seg)
        b.close()
        return g

    ref = grad(cme.FP64, 1, 5)
    one = grad(cme.FP32, 1, 5)
    got = grad(cme.FP32, 4, segment)
    for key in ref:
        e1, eC = rel(one[key], ref[key]), rel(got[key], ref[key])
        assert eC <= max(4 * e1, 1e-6), (key, e1, eC)
