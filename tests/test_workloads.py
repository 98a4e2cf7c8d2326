"""The seeded synthetic inputs follow their stated recipes (CPU): counts, sizes and parameters
of each workload, the lower CW branch plus complex Gaussian noise of the stated RMS as the
initial field, reproducible seeds, and the Fig. 1 mapping of the normalised Eq. 2."""
import numpy as np

from oracle import closed_forms as cf
from paper_1307_3428_gb300 import workloads as wl


def check_cw_start(inst, noise):
    """Pumped mode on the lower CW branch (smallest root of the cubic), every other mode
    noise of RMS `noise` (E|z|^2 = noise^2)."""
    P = cf.cw_powers(inst.sigma, inst.A_in, inst.kappa[inst.N // 2], inst.kappa_ext, inst.g0)[0]
    D00 = cf.cw_field(P, inst.sigma, inst.A_in, inst.kappa[inst.N // 2], inst.kappa_ext, inst.g0)
    assert abs(inst.D0[inst.N // 2] - D00) <= 10 * noise
    rest = np.delete(inst.D0, inst.N // 2)
    return np.mean(np.abs(rest) ** 2)


def test_sweep512():
    w = wl.sweep512()
    assert len(w.instances) == 256 and w.h == 5e-4 and w.nsteps == 20000
    powers = []
    for b, inst in enumerate(w.instances):
        assert inst.N == 512
        assert inst.sigma == -2.0 + 12.0 * b / 255
        assert inst.A_in == 2.5 and inst.g0 == 1.0 and inst.kappa_ext == 0.5
        assert np.all(inst.kappa == 1.0)
        assert np.allclose(inst.omega, 0.01 * inst.mu.astype(float) ** 2, rtol=0, atol=1e-12)
        powers.append(check_cw_start(inst, 1e-6))
    assert abs(np.mean(powers) / 1e-12 - 1.0) < 0.02      # 256 x 511 samples of |z|^2
    assert np.array_equal(wl.sweep512().instances[7].D0, w.instances[7].D0)   # seeded
    sub = wl.sweep512(indices=[128])
    assert np.array_equal(sub.instances[0].D0, w.instances[128].D0)
    other = wl.sweep512(seed_offset=256)
    assert not np.array_equal(other.instances[0].D0, w.instances[0].D0)


def test_uneven_and_adjoint():
    w = wl.uneven()
    assert len(w.instances) == 256 and w.h == 2e-4 and w.nsteps == 50000
    sizes = [i.N for i in w.instances]
    for N in (256, 1024, 2048, 4096):
        assert sizes.count(N) == 64
    for inst in w.instances:
        assert 0.0 <= inst.sigma <= 8.0 and 1.5 <= inst.A_in.real <= 3.0
        mu = inst.mu.astype(float)
        assert np.allclose(inst.omega, 0.01 * mu ** 2 / 2 + 1e-4 * mu ** 3 / 6, rtol=1e-14)
    a = wl.adjoint4096()
    assert len(a.instances) == 16 and all(i.N == 4096 for i in a.instances)
    assert a.h == 2e-4 and a.nsteps == 10000
    T = wl.sech2_target(4096, 16)
    assert T.shape == (16, 4096) and np.all(np.isfinite(T))
    assert np.all(T <= 0.0 + 1e-12)                        # P_t <= 1, sech^2 <= 1


def test_plain64_and_octave():
    p = wl.plain64()
    (inst,) = p.instances
    assert inst.N == 64 and inst.sigma == 2.5 and inst.A_in == 2.0 and p.h == 1e-3
    assert np.allclose(inst.omega, 0.02 * inst.mu.astype(float) ** 2)
    assert abs(check_cw_start(inst, 1e-4) / 1e-8 - 1.0) < 0.5   # 63 samples
    o = wl.octave()
    (big,) = o.instances
    assert big.N == 1 << 17 and big.sigma == 4.0 and big.A_in == 3.0 and o.h == 1e-4
    mu = big.mu.astype(float)
    assert np.allclose(big.omega, 2e-4 * mu ** 2 / 2 - 4e-7 * mu ** 3 / 6, rtol=1e-14)


def test_fig1_mapping():
    """Eq. 2 onto the library's model: kappa = 2, g0 = 1, kappa_ext = 1, A_in = f0,
    sigma = 0, omega = Omega = -0.00625 mu^2, 201 physical modes of 256, tau~ = 128 pi."""
    w = wl.fig1()
    assert len(w.instances) == 4
    assert abs(w.h * w.nsteps - 128 * np.pi) < 1e-12
    for inst, f in zip(w.instances, (1.01, 1.2, 1.8, 4.0)):
        assert inst.N == 256 and inst.M == 201
        assert np.all(inst.kappa == 2.0) and inst.g0 == 1.0 and inst.kappa_ext == 1.0
        assert inst.sigma == 0.0 and abs(inst.A_in - f * np.sqrt(2.0)) < 1e-15
        assert np.allclose(inst.omega, -0.00625 * inst.mu.astype(float) ** 2)
        check_cw_start(inst, 1e-4)
