"""The discrete adjoint (cme_grad) against the oracle's adjoint and against central finite
differences of the GPU's own FP64 loss; checkpoint-segment invariance; the FP32 adjoint against
the FP64 one; the torch.autograd wrapper."""
import copy

import numpy as np
import pytest

import oracle
from paper_1307_3428_gb300 import cme
from paper_1307_3428_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()
    cme.load()


def target_for(N, seed):
    rng = np.random.default_rng(seed)
    return np.log10(rng.uniform(1e-4, 0.5, N))


def small_instance(N, seed):
    inst = wl.make_instance(N, 0.05, 0.01, 1.3, 1.4 + 0.2j, 0.05, seed=seed)
    return inst


def gpu_grad(insts, h, n, T, prec=cme.FP64, segment=0):
    b = cme.Batch([cme.Instance.from_workload(i) for i in insts], precision=prec)
    return b.grad(h, n, np.concatenate(T), segment=segment)


@pytest.mark.parametrize("N", [4, 8, 16, 64])
def test_grad_matches_oracle_adjoint(N):
    h, n = 0.02, 30
    insts = [small_instance(N, 30 + k) for k in range(3)]
    T = [target_for(N, 40 + k) for k in range(3)]
    g = gpu_grad(insts, h, n, T)
    for k, (inst, t) in enumerate(zip(insts, T)):
        o = oracle.log_spectrum_grad(inst, h, n, t)
        sl = slice(k * N, (k + 1) * N)
        assert abs(g["loss"][k] - o["loss"]) <= 1e-11 * abs(o["loss"])
        for key, ref in (("d_sigma", o["sigma"]), ("d_D2", o["D2"]), ("d_D3", o["D3"])):
            assert abs(g[key][k] - ref) <= 1e-9 * max(abs(ref), 1e-6 * abs(o["loss"])), key
        assert abs(g["d_A_in"][k] - o["A_in"]) <= 1e-9 * abs(o["A_in"])
        scale = np.max(np.abs(o["D0"]))
        assert np.max(np.abs(g["d_D0"][sl] - o["D0"])) <= 1e-9 * scale
        assert np.max(np.abs(g["d_omega"][sl] - o["omega"])) <= 1e-9 * np.max(np.abs(o["omega"]))
        assert np.max(np.abs(g["d_kappa"][sl] - o["kappa"])) <= 1e-9 * np.max(np.abs(o["kappa"]))


def test_segments_do_not_change_the_gradient():
    N, h, n = 64, 0.01, 37
    insts = [small_instance(N, 50)]
    T = [target_for(N, 51)]
    ref = gpu_grad(insts, h, n, T, segment=1)
    for seg in (0, 5, 37, 100):
        g = gpu_grad(insts, h, n, T, segment=seg)
        for k in ref:
            assert np.array_equal(g[k], ref[k]), (seg, k)


def test_grad_matches_central_differences_fp64():
    """N=256, 400 steps of the sweep-like dynamics; central differences of the GPU FP64 loss
    agree with the adjoint to 1e-6.  Steps are 1e-6 relative to each parameter's value (D2 =
    0.01, D3 = 1e-4 move omega at mu = 128 by D mu^2/2, D mu^3/6, so an absolute 1e-6 step in
    D3 would shift the edge resonances by 0.35) and the stencil is fourth order."""
    N, h, n = 256, 2e-3, 400
    inst = wl.make_instance(N, 0.01, 1e-4, 3.0, 2.0, 1e-3, seed=60)
    T = [target_for(N, 61)]
    g = gpu_grad([inst], h, n, T)
    mu = np.arange(N) - N // 2

    def loss(**kw):
        i2 = copy.deepcopy(inst)
        for k, v in kw.items():
            setattr(i2, k, v)
        return gpu_grad([i2], h, n, T)["loss"][0]

    checks = [("sigma", 3.0e-6, lambda s: loss(sigma=inst.sigma + s), g["d_sigma"][0]),
              ("D2", 1e-8, lambda s: loss(omega=inst.omega + s * mu ** 2 / 2), g["d_D2"][0]),
              ("D3", 1e-10, lambda s: loss(omega=inst.omega + s * mu ** 3 / 6), g["d_D3"][0]),
              ("Are", 2e-6, lambda s: loss(A_in=inst.A_in + s), g["d_A_in"][0].real),
              ("Aim", 2e-6, lambda s: loss(A_in=inst.A_in + 1j * s), g["d_A_in"][0].imag)]
    rng = np.random.default_rng(62)
    for r in range(3):
        v = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        v *= 1e-3 / np.linalg.norm(v)          # direction of the size of the noise floor
        checks.append((f"D0_{r}", 1e-6, lambda s, v=v: loss(D0=inst.D0 + s * v),
                       float(np.real(np.vdot(g["d_D0"], v)))))
    for name, e, f, ad in checks:
        fd = (8 * (f(e) - f(-e)) - (f(2 * e) - f(-2 * e))) / (12 * e)
        assert abs(fd - ad) <= 1e-6 * max(abs(fd), abs(ad)), (name, fd, ad)


def test_fp32_adjoint_close_to_fp64():
    """The FP32 adjoint (FP32 field and cotangents, FP64 parameter accumulators) against the
    FP64 one on fields whose modes all sit far above FP32 resolution.  (With noise-level modes
    -- |D_mu| ~ 1e-6 beside an O(1) pump mode -- the FP32 field itself carries errors of order
    1e-7 of the comb on those modes, so their log-power terms, and gradients weighted towards
    them such as dL/dD2, are only loosely determined in FP32; gradient checks use FP64.)"""
    N, h, n = 512, 5e-4, 300
    insts = [wl.random_instance(N, 75 + k, amp=0.3 * np.sqrt(64.0 / N), sigma=1.0 + k,
                                A_in=1.5, D2=0.02) for k in range(2)]
    T = [target_for(N, 70 + k) for k in range(2)]
    g64 = gpu_grad(insts, h, n, T, cme.FP64)
    g32 = gpu_grad(insts, h, n, T, cme.FP32)
    for key in ("d_sigma", "d_D2", "d_A_in"):
        a, b = np.asarray(g32[key]), np.asarray(g64[key])
        assert np.max(np.abs(a - b)) <= 1e-3 * np.max(np.abs(b)), key
    assert np.linalg.norm(g32["d_D0"] - g64["d_D0"]) <= 1e-3 * np.linalg.norm(g64["d_D0"])
    assert np.max(np.abs(g32["loss"] - g64["loss"])) <= 1e-5 * np.max(np.abs(g64["loss"]))


def test_torch_autograd_wrapper():
    import torch
    N, h, n, B = 16, 0.02, 20, 2
    insts = [small_instance(N, 80 + k) for k in range(B)]
    T = np.stack([target_for(N, 90 + k) for k in range(B)])
    f64 = lambda x: torch.tensor(np.asarray(x, dtype=np.float64), requires_grad=True)
    sigma = f64([i.sigma for i in insts])
    a_re = f64([complex(i.A_in).real for i in insts])
    a_im = f64([complex(i.A_in).imag for i in insts])
    D2 = f64([0.05] * B)
    D3 = f64([0.01] * B)
    d0r = f64(np.stack([i.D0.real for i in insts]))
    d0i = f64(np.stack([i.D0.imag for i in insts]))
    L = cme.log_spectrum_loss(sigma, a_re, a_im, D2, D3, d0r, d0i, kappa=1.0, kappa_ext=0.5,
                              g0=1.0, h=h, nsteps=n, target=T.reshape(-1))
    L.backward()
    ref = [oracle.log_spectrum_grad(i, h, n, t) for i, t in zip(insts, T)]
    assert abs(L.item() - sum(r["loss"] for r in ref)) <= 1e-10 * L.item()
    for b in range(B):
        assert abs(sigma.grad[b].item() - ref[b]["sigma"]) <= 1e-8 * max(1, abs(ref[b]["sigma"]))
        assert abs(D2.grad[b].item() - ref[b]["D2"]) <= 1e-8 * max(1, abs(ref[b]["D2"]))
        assert np.allclose(d0r.grad[b].numpy() + 1j * d0i.grad[b].numpy(), ref[b]["D0"],
                           rtol=1e-8, atol=1e-8 * np.abs(ref[b]["D0"]).max())
