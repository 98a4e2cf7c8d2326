"""The FP32 error model of the kernels' RK4IP update, on the CPU: FP32 arithmetic emulated with
complex64 numpy arrays and single-precision scipy.fft transforms, on one sweep instance over the
bench horizon (20000 steps of h = 5e-4), each variant against the FP64 Eq. 4 engine.

- The kernels' form: FP64-derived propagators E = exp(L h/2), e1 = expm1(L h/2),
  e2 = expm1(L h) rounded to FP32, the increments x2 = D + (e1 D + h/2 k1) ..., and the state
  kept as a compensated pair (hi, lo) updated by an exact two-sum.
- The same increments without the compensation word.
- The textbook RK4IP formula in FP32, D' = E (A_I + h/6 (k1 + 2 k2 + 2 k3)) + h/6 k4.

The compensated form stays near FP32 resolution, while the other two lose one to two orders of
magnitude: the reason the kernels carry the (hi, lo) pair.  The measured errors are written to
the test's output."""
import numpy as np
import pytest

from oracle import fft_engine
from paper_1307_3428_gb300 import workloads as wl

sf = pytest.importorskip("scipy.fft")


def test_compensated_fp32_update_tracks_fp64():
    w = wl.sweep512(indices=[128])
    inst = w.instances[0]
    N, h, n = inst.N, w.h, w.nsteps
    fb = fft_engine.Batch([inst])
    ref = fft_engine.rk4ip(fb, h, n)[0]

    c64 = lambda z: np.asarray(z).astype(np.complex64)
    f32 = np.float32
    L = fb.L[0]
    E, e1, e2 = c64(np.exp(0.5 * h * L)), c64(np.expm1(0.5 * h * L)), c64(np.expm1(h * L))
    hh, hf, h6 = f32(0.5 * h), f32(h), f32(h / 6.0)
    pump = np.zeros(N, np.complex64)
    pump[N // 2] = np.complex64(np.sqrt(inst.kappa_ext) * inst.A_in)
    gN = f32(inst.g0 / N)
    assert sf.ifft(pump).dtype == np.complex64   # single-precision transforms

    def F(x):
        a = sf.ifft(np.fft.ifftshift(x)) * f32(N)
        b = (np.abs(a) ** 2).astype(np.float32) * a
        return (1j * gN) * np.fft.fftshift(sf.fft(b)) + pump

    def increments(comp):
        hi, lo = c64(fb.D0[0]), np.zeros(N, np.complex64)
        for _ in range(n):
            xF = F(hi)
            k1 = E * xF
            S = E * k1
            x = hi + (e1 * hi + hh * k1)
            xF = F(x)
            S = S + f32(2) * (E * xF)
            x = hi + (e1 * hi + hh * xF)
            xF = F(x)
            Ek3 = E * xF
            S = S + f32(2) * Ek3
            x = hi + (e2 * hi + hf * Ek3)
            xF = F(x)
            d = e2 * hi
            if comp:
                d = d + e2 * lo
            d = d + h6 * (S + xF)
            if comp:   # exact two-sum of hi and (lo + d)
                y = lo + d
                s = hi + y
                bb = s - hi
                lo = (hi - (s - bb)) + (y - bb)
                hi = s
            else:
                hi = hi + d
        return hi.astype(np.complex128) + lo.astype(np.complex128)

    def textbook():
        D = c64(fb.D0[0])
        for _ in range(n):
            AI = E * D
            k1 = E * F(D)
            k2 = F(AI + hh * k1)
            k3 = F(AI + hh * k2)
            k4 = F(E * (AI + hf * k3))
            D = E * (AI + h6 * (k1 + f32(2) * k2 + f32(2) * k3)) + h6 * k4
        return D.astype(np.complex128)

    rel = lambda x: float(np.linalg.norm(x - ref) / np.linalg.norm(ref))
    e_comp, e_inc, e_text = rel(increments(True)), rel(increments(False)), rel(textbook())
    print(f"FP32 vs FP64 after {n} steps: compensated {e_comp:.2e}, increments without "
          f"compensation {e_inc:.2e}, textbook RK4IP {e_text:.2e}")
    assert e_comp <= 2e-7
    assert e_inc >= 10 * e_comp and e_text >= 10 * e_comp
    assert max(e_comp, e_inc, e_text) <= 1e-4
