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
    for r in range(8):
        v = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        v *= 1e-3 / np.linalg.norm(v)          # direction of the size of the noise floor
        checks.append((f"D0_{r}", 1e-6, lambda s, v=v: loss(D0=inst.D0 + s * v),
                       float(np.real(np.vdot(g["d_D0"], v)))))
    for name, e, f, ad in checks:
        fd = (8 * (f(e) - f(-e)) - (f(2 * e) - f(-2 * e))) / (12 * e)
        assert abs(fd - ad) <= 1e-6 * max(abs(fd), abs(ad)), (name, fd, ad)


def fd_tolerance(fd, ad, L, e, rel=1e-6, ulps=32):
    """Bound on |fd - ad| for a fourth-order central difference with step e of a loss of value
    L: rel relative, plus the rounding noise of the difference quotient.  The FP64 loss of two
    nearby runs differs by rounding of a few ulps of L (measured up to 13 ulps at N = 4096,
    10000 steps), and the stencil (8, -8, -1, 1) / 12 multiplies that by 1.5 / e: below
    ulps * ulp(L) * 1.5 / e no difference quotient resolves the derivative."""
    return rel * max(abs(fd), abs(ad)) + 1.5 * ulps * np.spacing(abs(L)) / e


def _power_losses(insts, h, n, T):
    """Per-instance loss sum_mu (log10(|D_mu|^2 + 1e-20) - T_mu)^2 of the GPU FP64 forward run
    (cme_step, then the power spectrum of cme_spectrum), all instances in one batch."""
    b = cme.Batch([cme.Instance.from_workload(i) for i in insts], precision=cme.FP64)
    b.step(h, n)
    P = b.split(b.spectrum(cme.POWER))
    b.close()
    return np.array([np.sum((np.log10(p + 1e-20) - t) ** 2) for p, t in zip(P, T)])


# instances of the N = 4096 gradient workload checked at its full size: the MI-closest one
# (index 13, largest CW gain -0.14) and two others
ADJ4096_SAMPLE = [13, 0, 7]


def test_grad_adjoint4096_full_horizon_matches_central_differences():
    """The gradient workload at its own size: N = 4096, 10000 RK4IP steps of h = 2e-4, FP64.
    The adjoint of three of its instances against fourth-order central differences of the GPU
    FP64 loss, within 1e-6 relative plus the rounding noise of the difference quotient
    (fd_tolerance); the perturbed runs are independent instances of one batch.

    Steps (reading 12a): sigma, |A_in| and every initial-field mode (eight seeded directions
    v = D0 * w, w complex Gaussian) enter smoothly and take 1e-5 relative; 1e-6 leaves the
    quotient at the loss's rounding noise where a derivative is small against L / parameter
    (instance 7's dL/dRe A_in = 3.7 beside L = 5e5: 5.6e-6 off at 1e-6, measured).  D2 and D3
    move the edge resonance by D2 mu^2/2 and D3 mu^3/6 times their steps (2.1e4 and 1.4e5 at
    mu = 2048), so their steps are 3e-7 and 1e-7 relative: over tau = 2 that is 0.013 and 0.029
    rad at the edge.  At 1e-6 relative the truncation error is 7e-7 (D2) and 3e-3 (D3); at
    1e-7 the D3 quotient meets the rounding noise (4.6e-5 of dL/dD3, 13 ulps of L), so D3 is
    resolved to about 1e-4 and no step gives 1e-6 in FP64 (measured on GB300 over steps
    1e-4 ... 1e-10).  The chain rule dL/dD3 = sum_mu dL/domega_mu mu^3/6 (likewise D2) holds to
    1e-12 of the sum of its terms' magnitudes."""
    w = wl.adjoint4096()
    N, h, n = 4096, w.h, w.nsteps
    insts = [w.instances[k] for k in ADJ4096_SAMPLE]
    Tall = wl.sech2_target(N, 16)
    T = [Tall[k] for k in ADJ4096_SAMPLE]
    g = gpu_grad(insts, h, n, T)
    mu = (np.arange(N) - N // 2).astype(np.float64)
    for k in range(len(insts)):
        om = g["d_omega"][k * N:(k + 1) * N]
        for key, wgt in (("d_D2", mu ** 2 / 2), ("d_D3", mu ** 3 / 6)):
            assert abs(g[key][k] - np.sum(om * wgt)) <= 1e-12 * np.sum(np.abs(om * wgt)), key
    rng = np.random.default_rng(4700)
    dirs = []   # (name, instance index, step, perturb(inst, s), adjoint value)
    for k, inst in enumerate(insts):
        sl = slice(k * N, (k + 1) * N)
        e_sig = 1e-5 * abs(inst.sigma)
        e_A = 1e-5 * abs(inst.A_in)
        dirs += [
            ("sigma", k, e_sig, lambda i, s: setattr(i, "sigma", i.sigma + s), g["d_sigma"][k]),
            ("Re A_in", k, e_A, lambda i, s: setattr(i, "A_in", i.A_in + s), g["d_A_in"][k].real),
            ("Im A_in", k, e_A, lambda i, s: setattr(i, "A_in", i.A_in + 1j * s),
             g["d_A_in"][k].imag),
            ("D2", k, 3e-7 * 0.01, lambda i, s: setattr(i, "omega", i.omega + s * mu ** 2 / 2),
             g["d_D2"][k]),
            ("D3", k, 1e-7 * 1e-4, lambda i, s: setattr(i, "omega", i.omega + s * mu ** 3 / 6),
             g["d_D3"][k]),
        ]
        for r in range(8):
            v = inst.D0 * (rng.standard_normal(N) + 1j * rng.standard_normal(N))
            dirs.append((f"D0 direction {r}", k, 1e-5,
                         lambda i, s, v=v: setattr(i, "D0", i.D0 + s * v),
                         float(np.real(np.vdot(g["d_D0"][sl], v)))))
    pert, tgt = [], []
    for name, k, e, f, _ in dirs:
        for s in (e, -e, 2 * e, -2 * e):
            i2 = copy.deepcopy(insts[k])
            f(i2, s)
            pert.append(i2)
            tgt.append(T[k])
    base = _power_losses(insts, h, n, T)
    for k in range(len(insts)):
        assert abs(base[k] - g["loss"][k]) <= 1e-12 * abs(base[k])
    L = _power_losses(pert, h, n, tgt).reshape(-1, 4)
    rows = []
    for (name, k, e, _, ad), (lp, lm, lp2, lm2) in zip(dirs, L):
        fd = (8 * (lp - lm) - (lp2 - lm2)) / (12 * e)
        tol = fd_tolerance(fd, ad, base[k], e)
        rows.append((ADJ4096_SAMPLE[k], name, fd, ad, abs(fd - ad) / max(abs(fd), abs(ad)),
                     tol / max(abs(fd), abs(ad)), abs(fd - ad) <= tol))
    for r in rows:
        print("adjoint4096 instance %d %-16s fd %.12e adjoint %.12e rel %.2e (bound %.1e) %s" % r)
    for r in rows:
        assert r[6], r


def test_grad_n256_200_steps_matches_oracle_adjoint():
    """N = 256, 200 RK4IP steps of h = 2e-3: the GPU FP64 gradient against the FP64 oracle's
    discrete adjoint (direct-sum RK4IP), stored by tests/golden/make_adjoint_n256.py (the
    oracle takes about 2 s per step at this size).  Loss to 1e-11, gradients to 1e-9."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "adjoint_n256.json")) as fh:
        doc = json.load(fh)
    r = doc["recipe"]
    insts = [wl.make_instance(r["N"], r["D2"], r["D3"], s["sigma"], complex(*s["A_in"]),
                              r["noise"], seed=s["seed"]) for s in r["instances"]]
    T = wl.sech2_target(r["N"], len(insts))
    g = gpu_grad(insts, r["h"], r["nsteps"], list(T))
    N = r["N"]
    for k, o in enumerate(doc["instances"]):
        sl = slice(k * N, (k + 1) * N)
        assert abs(g["loss"][k] - o["loss"]) <= 1e-11 * abs(o["loss"])
        for key, ref in (("d_sigma", o["sigma"]), ("d_D2", o["D2"]), ("d_D3", o["D3"])):
            assert abs(g[key][k] - ref) <= 1e-9 * max(abs(ref), 1e-6 * abs(o["loss"])), key
        A = complex(*o["A_in"])
        assert abs(g["d_A_in"][k] - A) <= 1e-9 * abs(A)
        D0 = np.array([complex(*z) for z in o["D0"]])
        assert np.max(np.abs(g["d_D0"][sl] - D0)) <= 1e-9 * np.max(np.abs(D0))
        om = np.array(o["omega"])
        assert np.max(np.abs(g["d_omega"][sl] - om)) <= 1e-9 * np.max(np.abs(om))
        ka = np.array(o["kappa"])
        assert np.max(np.abs(g["d_kappa"][sl] - ka)) <= 1e-9 * np.max(np.abs(ka))


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


# ---------------------------------------------------------------------------------------------
# The Strang split step's adjoint (cme_grad on a CME_STRANG batch)

def gpu_grad_strang(insts, h, n, T, prec=cme.FP64, segment=0, **kw):
    b = cme.Batch([cme.Instance.from_workload(i) for i in insts], precision=prec,
                  integrator=cme.STRANG, **kw)
    g = b.grad(h, n, np.concatenate(T), segment=segment)
    b.close()
    return g


def _assert_matches_oracle(g, insts, T, h, n, method, tol=1e-9):
    for k, (inst, t) in enumerate(zip(insts, T)):
        N = inst.N
        o = oracle.log_spectrum_grad(inst, h, n, t, method=method)
        sl = slice(k * N, (k + 1) * N)
        assert abs(g["loss"][k] - o["loss"]) <= 1e-11 * abs(o["loss"])
        for key, ref in (("d_sigma", o["sigma"]), ("d_D2", o["D2"]), ("d_D3", o["D3"])):
            assert abs(g[key][k] - ref) <= tol * max(abs(ref), 1e-6 * abs(o["loss"])), key
        assert abs(g["d_A_in"][k] - o["A_in"]) <= tol * abs(o["A_in"])
        assert np.max(np.abs(g["d_D0"][sl] - o["D0"])) <= tol * np.max(np.abs(o["D0"]))
        assert np.max(np.abs(g["d_omega"][sl] - o["omega"])) <= tol * np.max(np.abs(o["omega"]))
        assert np.max(np.abs(g["d_kappa"][sl] - o["kappa"])) <= tol * np.max(np.abs(o["kappa"]))


@pytest.mark.parametrize("N", [4, 8, 16, 64, 256])
def test_strang_grad_matches_oracle_adjoint(N):
    """FP64 Strang gradients against the oracle's discrete adjoint of the split step: loss to
    1e-11, every gradient to 1e-9 (N = 4 and 8: thread groups narrower than a warp; N = 256:
    several groups' worth of passes)."""
    h, n = 0.02, 30 if N <= 64 else 8
    insts = [small_instance(N, 130 + k) for k in range(3)]
    T = [target_for(N, 140 + k) for k in range(3)]
    g = gpu_grad_strang(insts, h, n, T)
    _assert_matches_oracle(g, insts, T, h, n, oracle.STRANG)


def test_strang_grad_padding_and_cluster_match_oracle_adjoint():
    """201 physical modes in a 256-point transform (the padding of Sec. 2), and N = 256 spread
    over 2-block thread-block clusters, both in FP64 against the oracle's Strang adjoint."""
    N, h, n = 256, 0.02, 6
    insts = [small_instance(N, 150 + k) for k in range(2)]
    for i in insts:
        i.M = 201
    T = [target_for(N, 160 + k) for k in range(2)]
    g = gpu_grad_strang(insts, h, n, T)
    _assert_matches_oracle(g, insts, T, h, n, oracle.STRANG)
    insts = [small_instance(N, 170 + k) for k in range(2)]
    T = [target_for(N, 180 + k) for k in range(2)]
    g = gpu_grad_strang(insts, h, n, T, cluster=2)
    _assert_matches_oracle(g, insts, T, h, n, oracle.STRANG)


def test_strang_segments_do_not_change_the_gradient():
    N, h, n = 64, 0.01, 37
    insts = [small_instance(N, 190)]
    T = [target_for(N, 191)]
    ref = gpu_grad_strang(insts, h, n, T, segment=1)
    for seg in (0, 5, 37, 100):
        g = gpu_grad_strang(insts, h, n, T, segment=seg)
        for k in ref:
            assert np.array_equal(g[k], ref[k]), (seg, k)


def test_strang_grad_matches_central_differences_fp64():
    """N = 4096 on 8-block clusters and N = 256 on one block, 400 Strang steps of the sweep-like
    dynamics: fourth-order central differences of the GPU FP64 loss agree with the adjoint to
    1e-6 relative plus the difference quotient's rounding noise (fd_tolerance).  Steps 1e-5
    relative to sigma, |A_in| and each initial-field mode (eight seeded directions), 1e-6
    relative to D2 and to D3 (1e-7 at N = 4096; see the N = 4096 RK4IP check).  dL/dsigma of
    the N = 4096 run is small (1e-8 of L / sigma), so it is resolved only to the noise."""
    for N, h, n in ((256, 2e-3, 400), (4096, 2e-4, 400)):
        inst = wl.make_instance(N, 0.01, 1e-4, 3.0, 2.0 - 0.3j, 1e-3, seed=200 + N)
        T = [target_for(N, 201 + N)]
        g = gpu_grad_strang([inst], h, n, T)
        mu = (np.arange(N) - N // 2).astype(np.float64)
        rng = np.random.default_rng(202)
        # D2 and D3 move the edge resonances by up to 0.01 * 2048^2 / 2 and 1e-4 * 2048^3 / 6
        # times their steps, so theirs are smaller (the run is 400 steps, tau = 0.08 at N = 4096)
        e_D3 = 1e-7 if N == 4096 else 1e-6
        dirs = [("sigma", 1e-5 * inst.sigma, lambda i, s: setattr(i, "sigma", i.sigma + s),
                 g["d_sigma"][0]),
                ("Re A_in", 1e-5 * abs(inst.A_in), lambda i, s: setattr(i, "A_in", i.A_in + s),
                 g["d_A_in"][0].real),
                ("Im A_in", 1e-5 * abs(inst.A_in), lambda i, s: setattr(i, "A_in", i.A_in + 1j * s),
                 g["d_A_in"][0].imag),
                ("D2", 1e-6 * 0.01, lambda i, s: setattr(i, "omega", i.omega + s * mu ** 2 / 2),
                 g["d_D2"][0]),
                ("D3", e_D3 * 1e-4, lambda i, s: setattr(i, "omega", i.omega + s * mu ** 3 / 6),
                 g["d_D3"][0])]
        for r in range(8):
            v = inst.D0 * (rng.standard_normal(N) + 1j * rng.standard_normal(N))
            dirs.append((f"D0 direction {r}", 1e-5, lambda i, s, v=v: setattr(i, "D0", i.D0 + s * v),
                         float(np.real(np.vdot(g["d_D0"], v)))))
        pert = []
        for _, e, f, _ in dirs:
            for s in (e, -e, 2 * e, -2 * e):
                i2 = copy.deepcopy(inst)
                f(i2, s)
                pert.append(i2)
        b = cme.Batch([cme.Instance.from_workload(i) for i in pert], precision=cme.FP64,
                      integrator=cme.STRANG)
        b.step(h, n)
        P = b.split(b.spectrum(cme.POWER))
        b.close()
        L = np.array([np.sum((np.log10(p + 1e-20) - T[0]) ** 2) for p in P]).reshape(-1, 4)
        rows = []
        for (name, e, _, ad), (lp, lm, lp2, lm2) in zip(dirs, L):
            fd = (8 * (lp - lm) - (lp2 - lm2)) / (12 * e)
            tol = fd_tolerance(fd, ad, g["loss"][0], e)
            rows.append((N, name, fd, ad, abs(fd - ad) / max(abs(fd), abs(ad)),
                         tol / max(abs(fd), abs(ad)), abs(fd - ad) <= tol))
        for r in rows:
            print("strang N=%d %-16s fd %.12e adjoint %.12e rel %.2e (bound %.1e) %s" % r)
        for r in rows:
            assert r[6], r


def test_strang_fp32_adjoint_close_to_fp64():
    """FP32 Strang gradients against FP64 on fields whose modes all sit far above FP32
    resolution (as for RK4IP), one block per instance and 4-block clusters.  dL/dsigma, dL/dD2
    and dL/dD3 are sums over modes of the L cotangent weighted by -1, mu^2/2 and mu^3/6, whose
    terms cancel (at N = 4096 dL/dsigma is 1e-2 of the sum of its terms' magnitudes): each is
    held to 1e-3 of that sum of magnitudes, the scale its FP32 rounding acts on, or of its own
    value, whichever is larger.  The field, A_in and loss gradients have no such cancellation."""
    for N, C in ((512, 1), (4096, 4)):
        mu = (np.arange(N) - N // 2).astype(np.float64)
        insts = [wl.random_instance(N, 210 + k, amp=0.3 * np.sqrt(64.0 / N), sigma=1.0 + k,
                                    A_in=1.5, D2=0.02) for k in range(2)]
        T = [target_for(N, 220 + k) for k in range(2)]
        g64 = gpu_grad_strang(insts, 5e-4, 300, T, cme.FP64)
        g32 = gpu_grad_strang(insts, 5e-4, 300, T, cme.FP32, cluster=C)
        for k in range(2):
            om = np.abs(g64["d_omega"][k * N:(k + 1) * N])
            for key, w in (("d_sigma", 1.0), ("d_D2", mu ** 2 / 2), ("d_D3", np.abs(mu) ** 3 / 6)):
                a, b = g32[key][k], g64[key][k]
                assert abs(a - b) <= 1e-3 * max(abs(b), np.sum(om * w)), (N, k, key, a, b)
        # dL/dA_in sums the pump mode's cotangent over all 600 half flows; at N = 4096 the FP32
        # field itself is 1.6e-5 from FP64 after these 300 steps (1.2e-6 at N = 512), and the
        # sum carries that (measured 2.3e-3 on GB300, 8e-6 at N = 512)
        a, b = np.asarray(g32["d_A_in"]), np.asarray(g64["d_A_in"])
        assert np.max(np.abs(a - b)) <= (1e-3 if N <= 512 else 1e-2) * np.max(np.abs(b))
        assert np.linalg.norm(g32["d_D0"] - g64["d_D0"]) <= 1e-3 * np.linalg.norm(g64["d_D0"])
        assert np.max(np.abs(g32["loss"] - g64["loss"])) <= 1e-5 * np.max(np.abs(g64["loss"]))


def test_strang_cluster_adjoint_agrees_with_one_block():
    """The Strang backward kernel on 4- and 8-block clusters (N = 2048, 4096) against one block
    per instance, FP64: the same gradient to 1e-9."""
    for N, C in ((2048, 4), (4096, 8)):
        insts = [wl.make_instance(N, 0.01, 1e-4, 2.0 + k, 2.0, 1e-3, seed=230 + k)
                 for k in range(2)]
        T = np.concatenate([target_for(N, 240 + k) for k in range(2)])
        g = {}
        for c in (1, C):
            b = cme.Batch([cme.Instance.from_workload(i) for i in insts], precision=cme.FP64,
                          integrator=cme.STRANG, radix=8, cluster=c)
            g[c] = b.grad(2e-4, 30, T, segment=7)
            b.close()
        for key in g[1]:
            a, r = np.asarray(g[C][key]), np.asarray(g[1][key])
            assert np.linalg.norm(a - r) <= 1e-9 * np.linalg.norm(r), (N, key)


@pytest.mark.parametrize("integ", [cme.RK4IP, cme.STRANG])
@pytest.mark.parametrize("prec", [cme.FP64, cme.FP32])
def test_stored_and_recomputed_schedules_agree(prec, integ):
    """cme_grad stores the whole trajectory where it fits the budget (cme_set_grad_memory, by
    default half the free device memory) and otherwise checkpoints and recomputes segments on
    a second stream.  With the same launch plan both run the same arithmetic in the same
    order: the gradients are identical, on one block per instance (N = 64, segments of 5
    steps over 37) and on 4-block clusters (N = 4096, whose FP32 backward kernel prefetches)."""
    for N, kw in ((64, {}), (4096, {"cluster": 4, "radix": 8})):
        insts = [wl.make_instance(N, 0.01, 1e-4, 1.5 + k, 2.0, 1e-3, seed=250 + k)
                 for k in range(2)]
        T = np.concatenate([target_for(N, 260 + k) for k in range(2)])
        out = {}
        for budget in (-1, 0):
            b = cme.Batch([cme.Instance.from_workload(i) for i in insts], precision=prec,
                          integrator=integ, **kw)
            b.set_grad_memory(budget)
            out[budget] = b.grad(5e-4, 37, T, segment=5)
            assert b.last_grad_schedule == ("stored" if budget else "checkpoint")
            fin = b.get_state()
            b.close()
            out[budget]["final"] = fin
        for key in out[0]:
            assert np.array_equal(out[-1][key], out[0][key]), (N, key)
