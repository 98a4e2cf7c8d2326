"""Host-side checks of the shared-memory layouts of the in-block Stockham exchanges, with the
kernels' address arithmetic restated (the transform code of csrc/cme_core.cuh):

- padded layout p -> p + (p >> 4): every exchange address is a per-thread base plus a
  compile-time offset, pad(b + jL) = pad(b) + jL + (jL >> 4) for the write base
  b = (t - k) R + k, k = t mod L, and pad(t + jP) = pad(t) + jP + (jP >> 4) for the reads,
  at every N and values per thread R the kernels compile;
- XOR layout p -> p ^ (8 bit6(p)) of the exchange after a radix-8 pass of stride 8: the two
  per-thread bases of the kernels give exactly that map, it is a bijection, and each
  half-warp's writes and reads hit 16 distinct 8-byte banks;
- the passes themselves (butterfly slots, twiddle indices, exchange positions) compose to the
  unnormalised inverse DFT for every compiled transform shape.
CPU only."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1307_3428_gb300", "csrc")


def _macro_pairs(path, name):
    text = open(path).read()
    body = text[text.index("#define " + name):]
    body = body[:body.index("\n\n")]
    return [tuple(int(v) for v in m) for m in re.findall(r"X\(([\d, ]+)\)", body)
            for m in [m.split(",")]]


def compiled_transforms():
    """(log2 N, R) of every in-block transform the kernels instantiate: the one-block shapes,
    the block transforms of the cluster shapes (N / C points) and the rows and columns of
    the four-step large-N kernels."""
    launch = os.path.join(CSRC, "cme_launch.cuh")
    shapes = set(_macro_pairs(launch, "CME_FOR_EACH_SHAPE(X)"))
    for logn, r, c in _macro_pairs(launch, "CME_FOR_EACH_CLUSTER_SHAPE(X)"):
        shapes.add((logn - (c.bit_length() - 1), r))
    text = open(os.path.join(CSRC, "kern_large_fp32.cu")).read()
    first = text[text.index("#define"):]
    first = first[:first.index("\n\n")]
    shapes.update((int(a), int(b)) for a, b in re.findall(r"X\((\d+), (\d+)\)", first))
    return sorted(shapes)


def plan(logn, r):
    logr = r.bit_length() - 1
    n = 1 << logn
    p = n // r
    ns = (logn + logr - 1) // logr
    return n, p, ns, logr


def pad(p):
    return p + (p >> 4)


def test_shape_lists_parse():
    shapes = compiled_transforms()
    assert (9, 8) in shapes and (6, 2) in shapes and (12, 16) in shapes and (9, 4) in shapes
    assert all(2 <= r <= 16 and (1 << logn) >= r for logn, r in shapes)


@pytest.mark.parametrize("logn,r", [(n, r) for n in range(2, 13) for r in (2, 4, 8, 16)
                                    if (1 << n) >= r])
def test_padding_identity(logn, r):
    """Every (N, R) with N = 4 ... 4096, R = 2 ... 16: a superset of the compiled shapes."""
    n, p, ns, logr = plan(logn, r)
    for s in range(ns - 1):
        L = 1 << (s * logr)
        for t in range(p):
            k = t & (L - 1)
            b = (t - k) * r + k
            for j in range(r):
                assert pad(b + j * L) == pad(b) + j * L + ((j * L) >> 4), (s, t, j)
    for t in range(p):
        for j in range(r):
            assert pad(t + j * p) == pad(t) + j * p + ((j * p) >> 4), (t, j)


def xor8(p):
    return p ^ (8 * ((p >> 6) & 1))


@pytest.mark.parametrize("logn", [n for n, r in compiled_transforms() if r == 8
                                  and plan(n, 8)[2] >= 3 and plan(n, 8)[1] >= 16])
def test_xor_layout_of_the_stride_8_exchange(logn):
    n, p, _, _ = plan(logn, 8)
    assert sorted(xor8(q) for q in range(n)) == list(range(n))          # a bijection
    for t in range(p):
        c = (t >> 3) & 1
        wb = 64 * (t >> 3) + (t & 7)
        wx0, wx1 = wb + 8 * c, wb - 8 * c
        rx0 = t ^ (8 * ((t >> 6) & 1))
        rx1 = rx0 ^ 8
        for j in range(8):
            # the write of logical position b + 8 j, b = 64 (t >> 3) + (t & 7) (stride L = 8)
            assert (wx1 if j & 1 else wx0) + 8 * j == xor8(wb + 8 * j), (t, j)
            # the read of logical position t + j P
            assert (rx1 if ((j * p) >> 6) & 1 else rx0) + j * p == xor8(t + j * p), (t, j)
    for h in range(p // 16):
        ts = range(16 * h, 16 * h + 16)
        for j in range(8):
            writes = {xor8(64 * (t >> 3) + (t & 7) + 8 * j) % 16 for t in ts}
            reads = {xor8(t + j * p) % 16 for t in ts}
            assert len(writes) == 16 and len(reads) == 16, (h, j)


@pytest.mark.parametrize("logn,r", compiled_transforms())
def test_stockham_passes_and_twiddles(logn, r):
    """The in-block transform as the kernels run it: thread t holds positions t + j P; pass s
    (radix r_s, stride L = R^s, Q = R / r_s butterflies a thread) takes butterfly q from slots
    q + j Q, multiplies element j by the table entry (j k N / (L r_s)) mod N with
    k = (t + q P) mod L (exp(2 pi i j k / (L r_s))), runs the r_s-point transform, and (except
    after the last pass) writes slot j to position (t - k) R + k + j L and reads back t + j P.
    The result, in positions t + j P, is the unnormalised inverse DFT."""
    n, p, ns, logr = plan(logn, r)
    log_last = logn - (ns - 1) * logr
    tw = np.exp(2j * np.pi * np.arange(n) / n)
    X = np.array([1, 1j]) @ np.random.default_rng(logn * 17 + r).standard_normal((2, n))
    x = np.array([[X[t + j * p] for j in range(r)] for t in range(p)])
    for s in range(ns):
        rs = r if s < ns - 1 else 1 << log_last
        Q, L = r // rs, 1 << (s * logr)
        stride = n // (L * rs)
        for t in range(p):
            for q in range(Q):
                v = x[t, q + Q * np.arange(rs)]
                if s > 0:
                    k = (t + q * p) & (L - 1)
                    idx = (np.arange(rs) * k * stride) % n
                    # the table-read variant (large N): k_s = (t mod L) N / (L r_s) per pass,
                    # and butterflies q > 0 only in the last pass, where k = t + q P exactly
                    kst = (t & (L - 1)) * stride
                    assert np.array_equal(idx, (np.arange(rs) * kst
                                                + np.arange(rs) * q * p * stride) % n)
                    v = v * tw[idx]
                x[t, q + Q * np.arange(rs)] = rs * np.fft.ifft(v)
        if s + 1 < ns:
            buf = np.full(n, np.nan + 0j)
            for t in range(p):
                k = t & (L - 1)
                pos = (t - k) * r + k + np.arange(r) * L
                assert np.all(np.isnan(buf[pos]))
                buf[pos] = x[t]
            x = np.array([[buf[t + j * p] for j in range(r)] for t in range(p)])
    out = np.empty(n, complex)
    for t in range(p):
        out[t + p * np.arange(r)] = x[t]
    ref = n * np.fft.ifft(X)
    assert np.max(np.abs(out - ref)) <= 1e-9 * np.max(np.abs(ref))
