"""Host-side simulation of the large-N four-step transforms (N = N1 N2 > 4096, the row and
column kernels of csrc/cme_large.cuh), with the kernels' addresses restated, checked against
numpy's DFT:

- column pass, column m2: thread t, value j holds m1 (or j1) = t + j P1 of the column; the
  modes to time direction transforms over m1, multiplies by exp(+2 pi i j1 m2 / N) and stores
  Y at m2 N1 + t + j P1 (column-major, contiguous); the time to modes direction loads
  Z at t N2 + m2 + j P1 N2 and transforms over j1 into mode m1 N2 + m2;
- row pass, row j1: loads Y at t N1 + j1 + j P2 N1 (m2 = t + j P2), transforms over m2 into
  the time sample j1 + N1 (t + j P2); the time to modes direction transforms over j2,
  multiplies by exp(-2 pi i j1 m2 / N) and stores Z at j1 N2 + t + j P2 (row-major).
Every Y and Z position is written exactly once.  The in-block transforms are numpy's here (the
one-block transform code is checked element by element on the GPU).  CPU only."""
import numpy as np
import pytest


def split(logn):
    return logn - logn // 2, logn // 2          # N1 = 2^ceil(log N / 2), N2 = 2^floor(log N / 2)


def block(v, sign):
    """Transform of one row or column in local order: sign +1 unnormalised inverse DFT."""
    n = v.shape[-1]
    return n * np.fft.ifft(v, axis=-1) if sign > 0 else np.fft.fft(v, axis=-1)


@pytest.mark.parametrize("logn,R", [(13, 8), (14, 8), (16, 4), (17, 8), (17, 4)])
def test_four_step_index_maps(logn, R):
    l1, l2 = split(logn)
    N1, N2 = 1 << l1, 1 << l2
    N = N1 * N2
    P1, P2 = N1 // R, N2 // R
    rng = np.random.default_rng(logn * 10 + R)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    tw = np.exp(2j * np.pi * np.arange(N) / N)   # the table exp(2 pi i k / N)

    t1 = np.arange(P1)[:, None]
    t2 = np.arange(P2)[:, None]
    jj = np.arange(R)[None, :]

    # modes to time samples: column pass over every m2, then row pass over every j1
    Y = np.full(N, np.nan + 0j)
    for m2 in range(N2):
        m1 = t1 + jj * P1                              # (thread, value) -> m1
        col = np.empty(N1, complex)
        col[m1] = x[m1 * N2 + m2]
        out = block(col, +1)                           # local order j1 = t + j P1
        j1 = t1 + jj * P1
        addr = m2 * N1 + t1 + jj * P1
        assert np.all(np.isnan(Y[addr]))
        Y[addr] = out[j1] * tw[(j1 * m2) % N]
    assert not np.any(np.isnan(Y))
    a = np.full(N, np.nan + 0j)
    for j1 in range(N1):
        row = np.empty(N2, complex)
        m2 = t2 + jj * P2
        row[m2] = Y[t2 * N1 + j1 + jj * P2 * N1]
        out = block(row, +1)
        a[j1 + N1 * (t2 + jj * P2)] = out[t2 + jj * P2]
    ref = N * np.fft.ifft(x)
    assert np.max(np.abs(a - ref)) <= 1e-9 * np.max(np.abs(ref))

    # time samples to modes: row pass over every j1, then column pass over every m2
    b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    Z = np.full(N, np.nan + 0j)
    for j1 in range(N1):
        row = b[j1 + N1 * np.arange(N2)]               # j2 = 0 ... N2 - 1
        out = block(row, -1)
        m2 = t2 + jj * P2
        addr = j1 * N2 + t2 + jj * P2
        assert np.all(np.isnan(Z[addr]))
        Z[addr] = out[m2] * np.conj(tw[(j1 * m2) % N])
    assert not np.any(np.isnan(Z))
    X = np.full(N, np.nan + 0j)
    for m2 in range(N2):
        col = np.empty(N1, complex)
        j1 = t1 + jj * P1
        col[j1] = Z[t1 * N2 + m2 + jj * P1 * N2]
        out = block(col, -1)
        m1 = t1 + jj * P1
        X[m1 * N2 + m2] = out[m1]
    ref = np.fft.fft(b)
    assert np.max(np.abs(X - ref)) <= 1e-9 * np.max(np.abs(ref))
