"""The four-step path for N > 4096 (transforms split into N2 column transforms of length N1 and
N1 row transforms of length N2): transforms against the library transform numpy.fft, the
right-hand side and RK4IP runs against the oracle's Eq. 4 engine (pinned to the direct sum),
and the 2^17-mode octave workload."""
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


def batch_of(insts, prec, **kw):
    return cme.Batch([cme.Instance.from_workload(i) for i in insts], precision=prec, **kw)


LARGE = [8192, 16384, 65536, 131072]


@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
@pytest.mark.parametrize("N", LARGE)
def test_large_transform(N, prec):
    insts = [wl.random_instance(N, 2000 + k, amp=0.3 * np.sqrt(64.0 / N)) for k in range(2)]
    b = batch_of(insts, prec)
    got = b.split(b.transform(+1))
    for g, inst in zip(got, insts):
        ref = np.fft.ifft(np.fft.ifftshift(inst.D0)) * N     # a_j = sum_mu D_mu e^{+2 pi i j mu/N}
        tol = 1e-13 if prec == cme.FP64 else 2e-6
        assert np.max(np.abs(g - ref)) <= tol * np.max(np.abs(ref)) * np.log2(N)


@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
@pytest.mark.parametrize("N", [8192, 131072])
def test_large_rhs(N, prec):
    insts = [wl.random_instance(N, 2100 + k, amp=0.3 * np.sqrt(64.0 / N), A_in=1.1 - 0.2j)
             for k in range(2)]
    b = batch_of(insts, prec)
    got = b.split(b.eval_rhs())
    for g, inst in zip(got, insts):
        ref = fft_engine.Batch([inst]).F(inst.D0[None, :])[0]
        tol = 1e-12 if prec == cme.FP64 else 3e-6
        assert np.max(np.abs(g - ref)) <= tol * np.max(np.abs(ref)) * np.log2(N)


@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
@pytest.mark.parametrize("N", [8192, 32768])
def test_large_rk4ip_short(N, prec):
    insts = [wl.make_instance(N, 1e-3, 1e-6, 2.0 + k, 2.0, 1e-4, seed=2200 + k) for k in range(2)]
    b = batch_of(insts, prec)
    b.step(2e-4, 75)   # two whole 32-step graph chunks and a remainder
    got = b.split(b.get_state())
    refs = fft_engine.rk4ip(fft_engine.Batch(insts), 2e-4, 75)
    for g, r in zip(got, refs):
        assert rel(g, r) <= (1e-12 if prec == cme.FP64 else 1e-5)


def test_octave_workload():
    """N = 2^17, one instance: 1000 steps against the FP64 oracle (Eq. 4 engine); the full
    10000-step horizon in FP32 against the GPU's FP64 result; finite, status clean."""
    w = wl.octave()
    inst = w.instances[0]
    b32 = batch_of([inst], cme.FP32)
    b64 = batch_of([inst], cme.FP64)
    b32.step(w.h, 1000)
    b64.step(w.h, 1000)
    ref = fft_engine.rk4ip(fft_engine.Batch([inst]), w.h, 1000)[0]
    assert rel(b64.get_state(), ref) <= 1e-10
    assert rel(b32.get_state(), ref) <= 1e-4
    b32.step(w.h, w.nsteps - 1000)
    b64.step(w.h, w.nsteps - 1000)
    b32.synchronize()
    b64.synchronize()
    f32, f64 = b32.get_state(), b64.get_state()
    assert np.all(np.isfinite(f32)) and rel(f32, f64) <= 1e-4


def test_large_and_small_in_one_batch():
    insts = [wl.random_instance(256, 2300, amp=0.1),
             wl.random_instance(8192, 2301, amp=0.3 * np.sqrt(64.0 / 8192))]
    b = batch_of(insts, cme.FP64)
    b.step(1e-3, 40)
    for g, inst in zip(b.split(b.get_state()), insts):
        r = fft_engine.rk4ip(fft_engine.Batch([inst]), 1e-3, 40)[0]
        assert rel(g, r) <= 1e-12


@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
def test_largest_sizes(prec):
    """The top of the supported range: N = 2^20 (split 1024 x 1024) transform against
    numpy.fft, and N = 2^19 (1024 x 512) RK4IP against the Eq. 4 engine."""
    N = 1 << 20
    inst = wl.random_instance(N, 2300, amp=0.3 * np.sqrt(64.0 / N))
    b = batch_of([inst], prec)
    got = b.transform(+1)
    ref = np.fft.ifft(np.fft.ifftshift(inst.D0)) * N
    tol = 1e-13 if prec == cme.FP64 else 2e-6
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref)) * np.log2(N)
    b.close()
    N = 1 << 19
    insts = [wl.make_instance(N, 1e-4, 0.0, 2.0, 2.0, 1e-4, seed=2310)]
    b = batch_of(insts, prec)
    b.step(1e-4, 10)
    got = b.get_state()
    ref = fft_engine.rk4ip(fft_engine.Batch(insts), 1e-4, 10)[0]
    assert rel(got, ref) <= (1e-12 if prec == cme.FP64 else 1e-5)


@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
@pytest.mark.parametrize("N", [65536, 131072])
def test_four_values_per_thread(N, prec):
    """radix = 4 runs the row and column kernels at 4 values per thread (N1, N2 >= 256):
    transform against numpy.fft, and RK4IP against the Eq. 4 engine."""
    insts = [wl.random_instance(N, 2500 + k, amp=0.3 * np.sqrt(64.0 / N), D2=1e-4)
             for k in range(2)]
    b = batch_of(insts, prec, radix=4)
    got = b.split(b.transform(+1))
    for g, inst in zip(got, insts):
        ref = np.fft.ifft(np.fft.ifftshift(inst.D0)) * N
        tol = 1e-13 if prec == cme.FP64 else 2e-6
        assert np.max(np.abs(g - ref)) <= tol * np.max(np.abs(ref)) * np.log2(N)
    b.step(1e-4, 40)
    got = b.split(b.get_state())
    refs = fft_engine.rk4ip(fft_engine.Batch(insts), 1e-4, 40)
    for g, r in zip(got, refs):
        assert rel(g, r) <= (1e-12 if prec == cme.FP64 else 1e-5)


# FP32 four-step groups whose column blocks all fit on the GPU at once: (N, instances)
GRID_CASES = [(32768, 2), (65536, 2), (131072, 2), (262144, 1)]


@pytest.mark.parametrize("N,count", GRID_CASES)
def test_grid_kernel_matches_the_kernel_sequence_bitwise(N, count):
    """With persistent = 2 such groups run every step of a call in one kernel whose blocks
    meet at grid barriers (plan persistent 2, one launch per call); by default they run two
    kernels per RK stage.  The grid kernel repeats the row and column kernels' arithmetic
    expression for expression, so the two give the same bits: here with padding modes in one
    instance and per-mode Kerr coefficients in another, over 25 steps."""
    insts = [wl.make_instance(N, 1e-3, 1e-6, 2.0 + k, 2.0, 1e-4, seed=2600 + k)
             for k in range(count)]
    insts[0].M = (3 * N) // 4 + 1
    if count > 1:
        insts[1].g0_mu = wl.kerr_slope(1.0, N, 0.3)
    grid = batch_of(insts, cme.FP32, persistent=2)
    seq = batch_of(insts, cme.FP32)
    assert grid.plan(0)["persistent"] == 2 and seq.plan(0)["persistent"] == 1
    grid.step(2e-4, 25)
    seq.step(2e-4, 25)
    assert np.array_equal(grid.get_state(), seq.get_state())
    assert list(grid.status()) == [0] * count
    # a second call (propagators already computed for this h) is one launch, and continues
    # from the stored state
    grid.synchronize()
    n0 = cme.kernel_launches()
    grid.step(2e-4, 7)
    grid.synchronize()
    assert cme.kernel_launches() - n0 == 1
    seq.step(2e-4, 7)
    assert np.array_equal(grid.get_state(), seq.get_state())


def test_grid_barrier_wait_is_bounded():
    """Failure detection of the grid barriers without a device fault: the test switch
    (cme_debug_fault) makes every barrier expect one arrival more than there are blocks, so
    each block's poll runs out; the kernel finishes, the instance reports status 2,
    cme_synchronize returns TIMEOUT, and the batch then steps correctly again."""
    N = 32768
    inst = wl.make_instance(N, 1e-3, 1e-6, 2.5, 2.0, 1e-4, seed=2650)
    b = batch_of([inst], cme.FP32, persistent=2)
    assert b.plan(0)["persistent"] == 2
    D0 = b.get_state()
    b.debug_fault(1)
    b.step(2e-4, 3)
    with pytest.raises(cme.CmeError) as e:
        b.synchronize()
    assert e.value.code == -5
    assert list(b.status()) == [2]
    b.debug_fault(0)
    b.set_state(D0)
    b.step(2e-4, 10)
    b.synchronize()
    assert list(b.status()) == [0]
    ref = fft_engine.rk4ip(fft_engine.Batch([inst]), 2e-4, 10)[0]
    assert rel(b.get_state(), ref) <= 1e-5
