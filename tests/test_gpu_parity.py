"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: FP64 batches agree with the oracle to 1e-10 relative L2 of the final field; FP32
batches to 1e-4 (the stated bound for the FP32-field / FP64-propagator path).  Hot-path pieces
(transforms, the right-hand side) are compared element by element at tighter bounds."""
import os

import numpy as np
import pytest

import oracle
from oracle import closed_forms as cf
from oracle import fft_engine
from paper_1307_3428_gb300 import cme
from paper_1307_3428_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {cme.FP64: 1e-10, cme.FP32: 1e-4}
SIZES = [4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096]


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


# ---------------------------------------------------------------------------- hot-path pieces

@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
@pytest.mark.parametrize("N", SIZES)
def test_transform_matches_naive_dft(N, prec):
    insts = [wl.random_instance(N, 500 + k) for k in range(3)]
    b = batch_of(insts, prec)
    for sign in (+1, -1):
        got = b.split(b.transform(sign))
        for g, inst in zip(got, insts):
            if sign > 0:
                ref = oracle.dft(inst.D0, +1)
            else:  # sum_mu D_mu e^{-2 pi i j mu/N}: the +1 transform of the mirrored field
                ref = np.conj(oracle.dft(np.conj(inst.D0), +1))
            tol = 1e-13 if prec == cme.FP64 else 2e-6
            assert np.max(np.abs(g - ref)) <= tol * np.max(np.abs(ref)) * max(1, np.log2(N)), (sign,)


@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
@pytest.mark.parametrize("N", [4, 8, 16, 32, 64, 128, 256])
def test_rhs_matches_direct_sum(N, prec):
    insts = [wl.random_instance(N, 700 + k, A_in=1.1 - 0.3j * k, g0=0.5 + 0.25 * k)
             for k in range(3)]
    b = batch_of(insts, prec)
    got = b.split(b.eval_rhs())
    for g, inst in zip(got, insts):
        ref = oracle.rhs(inst.D0, inst.g0, inst.kappa_ext, inst.A_in)
        tol = 1e-12 if prec == cme.FP64 else 3e-6
        assert np.max(np.abs(g - ref)) <= tol * np.max(np.abs(ref)) * max(1, np.log2(N))


def test_rhs_n512_direct_sum_fp64():
    inst = wl.sweep512(indices=[37]).instances[0]
    b = batch_of([inst], cme.FP64)
    got = b.eval_rhs()
    ref = oracle.rhs(inst.D0, inst.g0, inst.kappa_ext, inst.A_in)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


# ---------------------------------------------------------------------------- integrators

@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
def test_plain_n64_full_horizon(prec):
    """N=64, one instance, h=1e-3, 2000 RK4IP steps against the direct-sum oracle."""
    w = wl.plain64()
    inst = w.instances[0]
    b = batch_of([inst], prec)
    b.step(w.h, w.nsteps)
    b.synchronize()
    got = b.get_state()
    ref = oracle.integrate(inst, w.h, w.nsteps, oracle.RK4IP)
    err = rel(got, ref)
    assert err <= TOL[prec], err
    # the power spectrum too
    assert rel(b.spectrum(cme.POWER), np.abs(ref) ** 2) <= TOL[prec]


@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
@pytest.mark.parametrize("N", SIZES)
def test_rk4ip_every_size_short(N, prec):
    """Random fields on all modes (every mode of the comb active), 20 steps, ragged batch."""
    amp = 0.3 * min(1.0, np.sqrt(64.0 / N))       # keeps |a_j|^2 = O(1) at every N
    insts = [wl.random_instance(N, 900 + k, amp=amp, sigma=0.5 * k, A_in=1.0 + 0.2j * k)
             for k in range(5)]
    b = batch_of(insts, prec)
    b.step(1e-3, 20)
    got = b.split(b.get_state())
    if N <= 64:
        refs = [oracle.integrate(i, 1e-3, 20, oracle.RK4IP) for i in insts]
    else:
        refs = fft_engine.rk4ip(fft_engine.Batch(insts), 1e-3, 20)
    for g, r in zip(got, refs):
        assert rel(g, r) <= (1e-12 if prec == cme.FP64 else 1e-5)


@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
@pytest.mark.parametrize("N", [4, 16, 64, 512])
def test_strang_matches_oracle(N, prec):
    amp = 0.3 * min(1.0, np.sqrt(64.0 / N))
    insts = [wl.random_instance(N, 1100 + k, amp=amp, sigma=1.0 + k, A_in=1.2) for k in range(3)]
    b = batch_of(insts, prec, cme.STRANG)
    b.step(2e-3, 200)
    got = b.split(b.get_state())
    if N <= 16:
        refs = [oracle.integrate(i, 2e-3, 200, oracle.STRANG) for i in insts]
    else:
        refs = fft_engine.strang(fft_engine.Batch(insts), 2e-3, 200)
    for g, r in zip(got, refs):
        assert rel(g, r) <= (1e-11 if prec == cme.FP64 else 1e-5)


def test_strang_merged_linear_flows():
    """The step kernels merge the linear half flows between consecutive Strang steps into one
    flow over h; a call of n steps then equals n calls of one step (each its own half flows, as
    the oracle takes them) to rounding: 1e-13 in FP64 over 150 steps, with the pump on, and
    with padding modes; chunked launches (steps_per_launch) and the cluster kernel likewise."""
    insts = [wl.random_instance(64, 1150 + k, amp=0.3, sigma=1.0 + k, A_in=1.4 - 0.3j)
             for k in range(3)]
    insts[1].M = 51
    merged = batch_of(insts, cme.FP64, cme.STRANG)
    merged.step(2e-3, 150)
    single = batch_of(insts, cme.FP64, cme.STRANG)
    for _ in range(150):
        single.step(2e-3, 1)
    ref = single.get_state()
    assert rel(merged.get_state(), ref) <= 1e-13
    chunked = batch_of(insts, cme.FP64, cme.STRANG, steps_per_launch=7)
    chunked.step(2e-3, 150)
    assert rel(chunked.get_state(), ref) <= 1e-13
    big = [wl.random_instance(2048, 1160 + k, amp=0.3 * np.sqrt(64.0 / 2048), A_in=1.2)
           for k in range(2)]
    ref = fft_engine.strang(fft_engine.Batch(big), 1e-3, 60)
    for kw in ({}, {"cluster": 4}):
        b = batch_of(big, cme.FP64, cme.STRANG, **kw)
        b.step(1e-3, 60)
        for g, r in zip(b.split(b.get_state()), ref):
            assert rel(g, r) <= 1e-11, kw


def test_strang_n64_direct_definition():
    w = wl.plain64(nsteps=300)
    inst = w.instances[0]
    for prec in (cme.FP64, cme.FP32):
        b = batch_of([inst], prec, cme.STRANG)
        b.step(w.h, w.nsteps)
        ref = oracle.integrate(inst, w.h, w.nsteps, oracle.STRANG)
        assert rel(b.get_state(), ref) <= TOL[prec]


def sweep_indices():
    # both ends, every MI-unstable instance (100 - 105, around sigma ~ 2.7 - 2.9, gains
    # 0.005 - 0.32), and a few in between
    return [0, 1, 57, 100, 101, 102, 103, 104, 105, 128, 200, 254, 255]


@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
def test_sweep512_full_batch_full_horizon(prec):
    """N=512 x 256 instances, 20000 RK4IP steps in the launch configuration of the benchmark
    (one graph replay); sampled instances against the FP64 oracle (Eq. 4 engine) at their
    comparison horizon (mi_horizon_steps: the largest MI gain of the sweep, 0.32, needs
    tau = 21 > 10 to raise the 1e-6 noise to 1e-3 of CW, so every sample is compared at the
    full horizon), every instance finite and status clean."""
    w = wl.sweep512()
    b = batch_of(w.instances, prec, use_graph=True)
    b.step(w.h, w.nsteps)
    b.synchronize()
    assert not b.status().any()
    got = b.split(b.get_state())
    idx = sweep_indices()
    for i in idx:
        assert mi_horizon_steps(w.instances[i], 512, 0.02, 0.0, w.h, w.nsteps, 1e-6) == w.nsteps
    sub = [w.instances[i] for i in idx]
    refs = fft_engine.rk4ip(fft_engine.Batch(sub), w.h, w.nsteps)
    errs = [rel(got[i], r) for i, r in zip(idx, refs)]
    assert max(errs) <= TOL[prec], errs
    for g in got:
        assert np.all(np.isfinite(g))


def test_sweep512_short_direct_sum():
    """Two instances of the sweep, 3 steps, against the direct O(N^3) definition."""
    w = wl.sweep512(indices=[3, 150])
    for prec in (cme.FP64, cme.FP32):
        b = batch_of(w.instances, prec)
        b.step(w.h, 3)
        got = b.split(b.get_state())
        for g, inst in zip(got, w.instances):
            ref = oracle.integrate(inst, w.h, 3, oracle.RK4IP)
            assert rel(g, ref) <= (1e-13 if prec == cme.FP64 else 1e-6)


# ---------------------------------------------------------------------------- launch paths

@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
def test_graph_chunking_and_packing_are_bitwise_identical(prec):
    insts = wl.sweep512(indices=range(0, 256, 23)).instances
    ref = batch_of(insts, prec)
    ref.step(5e-4, 60)
    base = ref.get_state()
    for kw in (dict(use_graph=True), dict(steps_per_launch=7), dict(inst_per_cta=2),
               dict(use_graph=True, steps_per_launch=25)):
        b = batch_of(insts, prec, **kw)
        b.step(5e-4, 60)
        assert np.array_equal(b.get_state(), base), kw


@pytest.mark.parametrize("radix", [4, 8])
def test_radix_variants_agree(radix):
    insts = wl.sweep512(indices=[10, 90, 180]).instances
    b = batch_of(insts, cme.FP64, radix=radix)
    b.step(5e-4, 50)
    refs = fft_engine.rk4ip(fft_engine.Batch(insts), 5e-4, 50)
    for g, r in zip(b.split(b.get_state()), refs):
        assert rel(g, r) <= 1e-12


@pytest.mark.parametrize("N", [64, 128])
def test_two_values_per_thread_fp64(N):
    """Small FP64 groups of N = 64, 128 take 2 values per thread by default (one warp per
    instance at N = 64: the shortest chain of FP64 instructions per thread); every values-per-
    thread choice agrees with the Eq. 4 engine, for RK4IP and Strang."""
    amp = 0.3 * min(1.0, np.sqrt(64.0 / N))
    insts = [wl.random_instance(N, 700 + k, amp=amp, sigma=0.4 * k, A_in=1.2 + 0.1j * k)
             for k in range(3)]
    assert batch_of(insts[:1], cme.FP64).plan(0)["radix"] == 2
    assert batch_of(insts[:1], cme.FP32).plan(0)["radix"] == 8
    for integ, engine in ((cme.RK4IP, fft_engine.rk4ip), (cme.STRANG, fft_engine.strang)):
        refs = engine(fft_engine.Batch(insts), 1e-3, 40)
        for radix in (2, 4, 8):
            b = batch_of(insts, cme.FP64, integ, radix=radix)
            b.step(1e-3, 40)
            for g, r in zip(b.split(b.get_state()), refs):
                assert rel(g, r) <= 1e-12, (integ, radix)


def test_narrow_groups_fill_no_more_warps_than_instances():
    """Groups narrower than a warp fill whole warps, but no more of them than the instances
    need: one N = 16 instance runs as one warp (16 groups of 2 threads, 15 of them surplus),
    and its result is bit for bit that of the same instance in a fuller block."""
    insts = [wl.random_instance(16, 500 + k, amp=0.3, sigma=0.3 * k, A_in=1.1) for k in range(40)]
    for prec in (cme.FP32, cme.FP64):
        one = batch_of(insts[:1], prec)
        p = one.plan(0)
        assert p["inst_per_cta"] * (16 // p["radix"]) == 32, p
        many = batch_of(insts, prec)
        assert many.plan(0)["inst_per_cta"] > p["inst_per_cta"]
        for b in (one, many):
            b.step(1e-3, 30)
        assert np.array_equal(one.get_state(), many.get_state()[:16]), prec


def test_uneven_sizes_in_one_batch():
    insts = [wl.random_instance(N, 1300 + N, amp=0.2 * min(1.0, np.sqrt(64.0 / N)))
             for N in (4, 16, 16, 64, 256, 256, 1024)]
    for prec in (cme.FP64, cme.FP32):
        b = batch_of(insts, prec)
        b.step(1e-3, 10)
        for g, inst in zip(b.split(b.get_state()), insts):
            r = fft_engine.rk4ip(fft_engine.Batch([inst]), 1e-3, 10)[0]
            assert rel(g, r) <= (1e-12 if prec == cme.FP64 else 1e-5)


def test_zero_steps_is_a_noop_and_bad_h_is_rejected():
    inst = wl.random_instance(32, 5)
    b = batch_of([inst], cme.FP64)
    s0 = b.get_state()
    b.step(1e-3, 0)
    assert np.array_equal(b.get_state(), s0)
    for h in (0.0, -1e-3, float("nan"), float("inf")):
        with pytest.raises(cme.CmeError) as e:
            b.step(h, 1)
        assert e.value.code == -1
    with pytest.raises(cme.CmeError):
        b.step(1e-3, -1)


def test_nonfinite_field_sets_status():
    good = wl.random_instance(16, 1)
    bad = wl.random_instance(16, 2, amp=1e200)   # overflows to inf within a few steps
    b = batch_of([good, bad, good], cme.FP64)
    b.step(1e-2, 5)
    st = b.status()
    assert st[0] == 0 and st[1] == 1 and st[2] == 0
    with pytest.raises(cme.CmeError) as e:
        b.synchronize()
    assert e.value.code == -4
    b.set_state(np.concatenate([good.D0, good.D0, good.D0]))
    assert not b.status().any()


def test_state_roundtrip_checkpoint_and_resume_bitwise():
    insts = wl.sweep512(indices=[5, 77]).instances
    for prec in (cme.FP64, cme.FP32):
        a = batch_of(insts, prec)
        a.step(5e-4, 40)
        blob = a.checkpoint()
        a.step(5e-4, 40)
        fin = a.get_state()
        b = batch_of(insts, prec)
        b.restore(blob)
        assert abs(b.time() - 40 * 5e-4) < 1e-15
        b.step(5e-4, 40)
        assert np.array_equal(b.get_state(), fin)
        # FP64 state export/import round trip
        s = a.get_state()
        a.set_state(s)
        assert np.array_equal(a.get_state(), s)


def test_eq1_frame_output():
    w = wl.plain64(nsteps=200)
    inst = w.instances[0]
    b = batch_of([inst], cme.FP64)
    b.step(w.h, w.nsteps)
    D = b.get_state()
    A = b.spectrum(cme.FIELD_EQ1)
    assert rel(A, oracle.to_lab_frame(inst, D, w.h * w.nsteps)) <= 1e-14
    assert rel(b.spectrum(cme.FIELD_D), D) == 0.0


def test_torch_allocator_and_stream():
    import torch
    cme.use_torch_allocator()
    try:
        s = torch.cuda.Stream()
        inst = wl.plain64(nsteps=100).instances[0]
        b = cme.Batch([cme.Instance.from_workload(inst)], precision=cme.FP64,
                      stream=s.cuda_stream)
        b.step(1e-3, 100)
        ref = oracle.integrate(inst, 1e-3, 100, oracle.RK4IP)
        assert rel(b.get_state(), ref) <= 1e-11
        b.close()
    finally:
        cme.load().cme_set_allocator(cme.ALLOC_FN(), cme.FREE_FN(), None)


# ---------------------------------------------------------------------------- uneven batches

def mi_horizon_steps(inst, N, D2, D3, h, nsteps, noise):
    """Steps at which an instance is compared with the oracle.  MI-stable instances (closed-form
    CW gain <= 0): the full horizon.  MI-unstable ones: the last step before the seeded
    perturbation, grown at the closed-form gain, reaches 1e-3 of the CW amplitude (beyond it
    round-off grows at the same rate, and parity is not meaningful), or the full horizon if
    that comes first."""
    P = cf.cw_powers(inst.sigma, inst.A_in, inst.kappa[N // 2], inst.kappa_ext, inst.g0)[0]
    gain = cf.max_mi_gain(P, N, D2, D3, inst.sigma, inst.kappa[N // 2], inst.g0)
    if gain <= 0:
        return nsteps
    tau = np.log(1e-3 * np.sqrt(P) / noise) / gain
    return int(min(nsteps, np.floor(tau / h)))


def uneven_sample_indices():
    """Indices into the uneven workload's 256 instances: the first 8 MI-stable instances of
    each N, and every MI-unstable one."""
    w = wl.uneven(nsteps=1)
    picks = []
    for k, N in enumerate((256, 1024, 2048, 4096)):
        stable = 0
        for b in range(64 * k, 64 * (k + 1)):
            inst = w.instances[b]
            P = cf.cw_powers(inst.sigma, inst.A_in, 1.0, 0.5, 1.0)[0]
            if cf.max_mi_gain(P, N, 0.01, 1e-4, inst.sigma, 1.0, 1.0) > 0:
                picks.append(b)
            elif stable < 8:
                picks.append(b)
                stable += 1
    return sorted(picks)


_uneven_refs = {}


def uneven_oracle_refs():
    """The Eq. 4 engine's results for the uneven sample, each at its comparison horizon,
    computed once per session on a spawn process pool (one instance per task)."""
    if not _uneven_refs:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        w = wl.uneven()
        jobs = []
        for i in uneven_sample_indices():
            inst = w.instances[i]
            n = mi_horizon_steps(inst, inst.N, 0.01, 1e-4, w.h, w.nsteps, 1e-6)
            jobs.append((i, n))
        # longest first, so that the N = 4096 runs do not start last
        jobs.sort(key=lambda j: -w.instances[j[0]].N * j[1])
        with ProcessPoolExecutor(max_workers=os.cpu_count() or 4,
                                 mp_context=mp.get_context("spawn")) as pool:
            res = pool.map(fft_engine.rk4ip_one, [(w.instances[i], w.h, n) for i, n in jobs])
            for (i, n), r in zip(jobs, res):
                _uneven_refs[i] = (n, r)
    return _uneven_refs


@pytest.mark.parametrize("persistent", [1, 2])
def test_uneven_modes_agree_bitwise_and_with_oracle(persistent):
    """Mixed N (4..4096) in one batch: the persistent work-list kernel and the concurrent
    per-group kernels agree (FP64: to 1e-14 -- the per-group plan may run other values per
    thread than the work-list tiles); both agree with the oracle."""
    sizes = (4, 8, 64, 64, 256, 512, 1024, 2048, 4096)
    insts = [wl.random_instance(N, 1500 + i, amp=0.2 * min(1.0, np.sqrt(64.0 / N)), sigma=1.0,
                                A_in=1.3) for i, N in enumerate(sizes)]
    for prec in (cme.FP64, cme.FP32):
        b = batch_of(insts, prec, persistent=persistent, use_graph=True)
        b.step(1e-3, 12)
        got = b.split(b.get_state())
        ref1 = batch_of(insts, prec, persistent=3 - persistent)
        ref1.step(1e-3, 12)
        if prec == cme.FP64:
            assert np.array_equal(b.get_state(), ref1.get_state()) or \
                rel(b.get_state(), ref1.get_state()) < 1e-14
        for g, inst in zip(got, insts):
            r = fft_engine.rk4ip(fft_engine.Batch([inst]), 1e-3, 12)[0]
            assert rel(g, r) <= (1e-12 if prec == cme.FP64 else 1e-5)


@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
def test_uneven_full_batch_full_horizon(prec):
    """N in {256, 1024, 2048, 4096} x 64 instances, 50000 RK4IP steps of h=2e-4 in one
    persistent launch (one graph) against the FP64 oracle (Eq. 4 engine): eight MI-stable
    instances per N and every MI-unstable one, each at its comparison horizon
    (mi_horizon_steps; the unstable instances of this workload have gains of 0.025 - 0.034,
    so their perturbations stay far below 1e-3 of CW up to tau = 10 and they too are compared
    at the full horizon).  Instances whose horizon is shorter run again to that step."""
    refs = uneven_oracle_refs()
    w = wl.uneven()
    b = batch_of(w.instances, prec, use_graph=True, persistent=2)
    b.step(w.h, w.nsteps)
    b.synchronize()
    assert not b.status().any()
    got = b.split(b.get_state())
    short = {i: n for i, (n, _) in refs.items() if n < w.nsteps}
    for n in sorted(set(short.values())):
        sel = [i for i, m in short.items() if m == n]
        bs = batch_of([w.instances[i] for i in sel], prec)
        bs.step(w.h, n)
        for i, g in zip(sel, bs.split(bs.get_state())):
            got[i] = g
    assert len(refs) >= 35
    for i, (n, ref) in refs.items():
        err = rel(got[i], ref)
        assert err <= TOL[prec], (i, w.instances[i].N, n, err)


def test_autotune_keeps_state_and_results():
    insts = wl.sweep512(indices=range(0, 256, 8)).instances
    for prec in (cme.FP32, cme.FP64):
        a = batch_of(insts, prec)
        s0 = a.get_state()
        plan = a.autotune(5e-4, probe_steps=40)
        assert plan["radix"] in (0, 4, 8, 16) and plan["persistent"] in (1, 2)
        assert np.array_equal(a.get_state(), s0)
        assert a.time() == 0.0
        a.step(5e-4, 30)
        ref = fft_engine.rk4ip(fft_engine.Batch(insts), 5e-4, 30)
        for g, r in zip(a.split(a.get_state()), ref):
            assert rel(g, r) <= TOL[prec]


def test_autotune_uneven():
    insts = [wl.random_instance(N, 1700 + i, amp=0.1) for i, N in enumerate((64, 256, 256, 1024))]
    b = batch_of(insts, cme.FP32)
    plan = b.autotune(1e-3, probe_steps=20)
    assert plan["persistent"] in (1, 2)
    b.step(1e-3, 10)
    for g, inst in zip(b.split(b.get_state()), insts):
        r = fft_engine.rk4ip(fft_engine.Batch([inst]), 1e-3, 10)[0]
        assert rel(g, r) <= 1e-5
