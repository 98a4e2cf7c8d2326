"""Host-side simulation of the four-step transform of an instance spread over the C blocks of
a thread-block cluster, with the kernels' index arithmetic restated (ClusterFFT, the cluster
all-to-all and the cluster set-up in csrc/cme_core.cuh and csrc/cme_step.cuh), checked against
numpy's DFT for every compiled cluster shape:

- modes: thread l of block r holds k = r + C (l + PC j), j < R (PC = P / C threads a block);
- modes to time samples: the N2-point block transform, the twiddle exp(2 pi i n2 k1 / N) of
  local position n2 = l + PC j (k1 = r), the all-to-all (value j of thread (r, l) lands at
  position l + PC (r G + j div C) of block j mod C, G = R / C), C-point transforms over the
  slots {c G + m}, after which thread l of block r holds n = r PC + l + j P;
- time samples to modes: the same stages in reverse (C-point transforms, the twiddle of
  n2 = r PC + l + P (j mod G), k1 = j div G, value j to position l + PC (r + C (j mod G)) of
  block j div G, the block transform).
The block transform itself is the one-block Stockham code, checked element by element on the
GPU; here it is numpy's.  Every receiving position is written exactly once.  CPU only."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def cluster_shapes():
    text = open(os.path.join(ROOT, "paper_1307_3428_gb300", "csrc", "cme_launch.cuh")).read()
    body = text[text.index("#define CME_FOR_EACH_CLUSTER_SHAPE(X)"):]
    body = body[:body.index("\n\n")]
    return [tuple(int(v) for v in m) for m in re.findall(r"X\((\d+), (\d+), (\d+)\)", body)]


def table(N):
    return np.exp(2j * np.pi * np.arange(N) / N)   # the twiddle table exp(2 pi i m / N)


def block_transform(xb, PC, R):
    """+i transform of N2 = PC R points; input and output at local index l + PC j of (l, j)."""
    N2 = PC * R
    v = np.empty(N2, complex)
    for l in range(PC):
        for j in range(R):
            v[l + PC * j] = xb[l][j]
    y = N2 * np.fft.ifft(v)
    return [[y[l + PC * j] for j in range(R)] for l in range(PC)]


def radix_c(x, C, G):
    """+i C-point transforms over the slots {c G + m : c < C}, m < G, in place."""
    for m in range(G):
        v = np.array([x[c * G + m] for c in range(C)])
        y = C * np.fft.ifft(v)
        for c in range(C):
            x[c * G + m] = y[c]


def all_to_all(x, C, PC, R, to_modes):
    G = R // C
    buf = [[None] * (R * PC) for _ in range(C)]
    for r in range(C):
        for l in range(PC):
            for j in range(R):
                if to_modes:
                    dst, pos = j // G, l + PC * (r + C * (j % G))
                else:
                    dst, pos = j % C, l + PC * (r * G + j // C)
                assert buf[dst][pos] is None, "position written twice"
                buf[dst][pos] = x[r][l][j]
    assert all(v is not None for b in buf for v in b), "position never written"
    return [[[buf[r][l + PC * s] for s in range(R)] for l in range(PC)] for r in range(C)]


@pytest.mark.parametrize("logn,R,C", cluster_shapes())
def test_cluster_four_step_transform(logn, R, C):
    N = 1 << logn
    P, PC, N2, G = N // R, N // R // C, N // C, R // C
    w = table(N)
    rng = np.random.default_rng(logn * 100 + C)
    X = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    ref = N * np.fft.ifft(X)   # a_n = sum_k X_k exp(+2 pi i n k / N)

    # modes to time samples
    x = [[[X[r + C * (l + PC * j)] for j in range(R)] for l in range(PC)] for r in range(C)]
    x = [block_transform(x[r], PC, R) for r in range(C)]
    for r in range(C):
        for l in range(PC):
            for j in range(R):
                x[r][l][j] *= w[((l + PC * j) * r) % N]
    x = all_to_all(x, C, PC, R, to_modes=False)
    for r in range(C):
        for l in range(PC):
            radix_c(x[r][l], C, G)
    got = np.empty(N, complex)
    for r in range(C):
        for l in range(PC):
            for j in range(R):
                got[r * PC + l + j * P] = x[r][l][j]
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))

    # time samples to modes: the +i transform of the samples, back in the mode layout
    Y = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    ref = N * np.fft.ifft(Y)
    y = [[[Y[r * PC + l + j * P] for j in range(R)] for l in range(PC)] for r in range(C)]
    for r in range(C):
        for l in range(PC):
            radix_c(y[r][l], C, G)
            tp = r * PC + l
            for j in range(R):
                y[r][l][j] *= w[((tp + P * (j % G)) * (j // G)) % N]
    y = all_to_all(y, C, PC, R, to_modes=True)
    y = [block_transform(y[r], PC, R) for r in range(C)]
    got = np.empty(N, complex)
    for r in range(C):
        for l in range(PC):
            for j in range(R):
                got[r + C * (l + PC * j)] = y[r][l][j]
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))
    assert N2 == G * P
