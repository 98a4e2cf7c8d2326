"""cme_rk4ip_noalloc: the FP64 RK4IP integration for callers that may not allocate device memory
themselves (an application that hands out all device memory from its own fixed pool, or code
that must not call cudaMalloc because it can synchronise the device).  Its scratch lives in a
fixed 16 MiB device array inside the library.

The test checks it against the ordinary batch path (cme_batch_create + cme_step, FP64 RK4IP)
on two calls in a row with different sizes and parameters -- the second call reuses the array
the first one left filled -- and that sizes beyond the array are refused.  This file is named
so that pytest collects it last."""
import numpy as np
import pytest

from paper_1307_3428_gb300 import cme
from paper_1307_3428_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()
    cme.load()


def _run_noalloc(insts, h, nsteps):
    """Inputs and the field live in caller-owned torch tensors; the library allocates nothing."""
    import torch
    N, count = insts[0].N, len(insts)
    dev = torch.device("cuda")
    kappa = torch.tensor(np.concatenate([i.kappa for i in insts]), dtype=torch.float64, device=dev)
    omega = torch.tensor(np.concatenate([i.omega for i in insts]), dtype=torch.float64, device=dev)
    inst = torch.tensor(np.array([[i.g0, i.kappa_ext, complex(i.A_in).real, complex(i.A_in).imag,
                                   i.sigma] for i in insts]).reshape(-1), dtype=torch.float64,
                        device=dev)
    field = torch.tensor(np.concatenate([i.D0 for i in insts]).view(np.float64).copy(),
                         dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    cme.rk4ip_noalloc(N, count, h, nsteps, kappa.data_ptr(), omega.data_ptr(), inst.data_ptr(),
                      field.data_ptr(), stream)
    torch.cuda.synchronize()
    return field.cpu().numpy().view(np.complex128)


def _run_batch(insts, h, nsteps, **kw):
    b = cme.Batch([cme.Instance.from_workload(i) for i in insts], precision=cme.FP64, **kw)
    b.step(h, nsteps)
    out = b.get_state()
    b.close()
    return out


def test_noalloc_matches_batch_path_on_two_calls():
    cases = [
        (wl.sweep512(indices=range(0, 256, 16)).instances, 5e-4, 400),
        ([wl.random_instance(64, 900 + k, amp=0.3, sigma=0.4 * k, A_in=1.2 + 0.1j * k)
          for k in range(5)], 1e-3, 300),
    ]
    for insts, h, n in cases:
        got = _run_noalloc(insts, h, n)
        ref = _run_batch(insts, h, n)
        N = insts[0].N
        for k in range(len(insts)):
            g, r = got[k * N:(k + 1) * N], ref[k * N:(k + 1) * N]
            err = np.linalg.norm(g - r) / np.linalg.norm(r)
            assert err <= TOL_FP64, (N, k, err)


@pytest.mark.parametrize("N,count", [(4, 3), (8, 5), (2048, 4), (4096, 3)])
def test_noalloc_launch_shape_is_the_batch_plan(N, count):
    """The smallest sizes (one thread group narrower than a warp: N = 4 at 4 values per thread,
    N = 8 at 8) and the sizes whose Runge-Kutta accumulator lives in shared memory in FP64
    (N = 2048, 4096).  The result is bit for bit that of a batch with one block per instance
    (the one-block plan the entry point shares with cme_batch_create), and within the FP64
    tolerance of the default batch, which spreads few N >= 2048 instances over thread-block
    clusters and so rounds in another order.  Each call counts its six kernels."""
    amp = 0.3 * min(1.0, np.sqrt(64.0 / N))
    insts = [wl.random_instance(N, 950 + k, amp=amp, sigma=0.3 * k, A_in=1.1 + 0.2j * k)
             for k in range(count)]
    before = cme.kernel_launches()
    got = _run_noalloc(insts, 1e-3, 60)
    assert cme.kernel_launches() - before == 6
    assert np.array_equal(got, _run_batch(insts, 1e-3, 60, cluster=1))
    ref = _run_batch(insts, 1e-3, 60)
    for k in range(count):
        g, r = got[k * N:(k + 1) * N], ref[k * N:(k + 1) * N]
        assert np.linalg.norm(g - r) <= TOL_FP64 * np.linalg.norm(r), (N, k)


def test_noalloc_does_not_report_nonfinite_results():
    """The entry point returns before its kernels run and reads nothing back, so a field that
    overflows comes back non-finite with CME_OK: the caller checks the field."""
    insts = [wl.random_instance(64, 990 + k, amp=0.3) for k in range(2)]
    insts[1].D0 = insts[1].D0 * 1e200          # |a|^2 a overflows in the first step
    got = _run_noalloc(insts, 1e-3, 3)
    assert np.all(np.isfinite(got[:64]))
    assert not np.all(np.isfinite(got[64:]))


def test_noalloc_refuses_sizes_beyond_its_array():
    import torch
    N, count = 4096, 64          # 262144 modes: more than the fixed array holds
    x = torch.zeros(2 * N * count, dtype=torch.float64, device="cuda")
    p = torch.zeros(5 * count, dtype=torch.float64, device="cuda")
    with pytest.raises(cme.CmeError) as e:
        cme.rk4ip_noalloc(N, count, 1e-3, 1, x.data_ptr(), x.data_ptr(), p.data_ptr(),
                          x.data_ptr())
    assert e.value.code == -1
    assert "scratch" in str(e.value)
