"""The index rule of the fused x pass of the plane transform, restated on the host (CPU only).

The plane pass's inverse x transform is a Stockham sequence of radix stages; its last stage
(radix R) leaves butterfly j holding outputs j + q N/R, q < R.  Those are exactly the inputs
that the first stage of a forward transform running the same radices in reverse order reads
for its butterfly j, and that first stage has no twiddles.  So the inverse's last stage, the
potential multiply and the forward's first stage can run on one thread's registers.  This
test runs that schedule with plain DFT butterflies for every transform length the kernels
ship and both radix orders, and compares it with numpy's FFT of the same product.  The GPU
parity tests check the kernels; this pins the rule they are built on."""
import numpy as np
import pytest

LENGTHS = (24, 32, 60, 72, 96, 144, 180, 288)


def factor(n, order):
    """Radix sequence: order 0 odd radices first (9, 3, 5, then 8, 4, 2); order 1 largest
    radix first (8, 9, 4, 3, 5, 2)."""
    r, m = [], n
    seq = (8, 9, 4, 3, 5, 8, 4, 2) if order == 1 else (9, 3, 5, 8, 4, 2)
    for R in seq:
        while m % R == 0:
            r.append(R)
            m //= R
    assert m == 1
    return r


def dft(x, sign):
    R = len(x)
    k = np.arange(R)
    return np.exp(sign * 2j * np.pi * np.outer(k, k) / R) @ x


def stage(a, N, R, NS, sign):
    """One Stockham stage: butterfly j reads a[j + r N/R], twiddles by W_{NS R}^{r k}
    (k = j mod NS) and writes its R outputs NS apart from (j / NS) NS R + k."""
    NB = N // R
    out = np.empty_like(a)
    for j in range(NB):
        k = j % NS
        x = np.array([a[j + r * NB] * np.exp(sign * 2j * np.pi * r * k / (NS * R)) for r in range(R)])
        y = dft(x, sign)
        d = (j // NS) * NS * R + k
        out[d + np.arange(R) * NS] = y
    return out


def fused(a, N, R, V):
    """The inverse's last stage (NS = N / R), the potential multiply and the reversed forward
    plan's first stage (NS = 1, no twiddles) on butterfly j's R values."""
    NB = N // R
    out = np.empty_like(a)
    for j in range(NB):
        x = np.array([a[j + r * NB] * np.exp(2j * np.pi * r * j / N) for r in range(R)])
        y = dft(x, +1) * V[j + np.arange(R) * NB]
        out[j * R + np.arange(R)] = dft(y, -1)
    return out


@pytest.mark.parametrize("N", LENGTHS)
@pytest.mark.parametrize("order", (0, 1))
def test_fused_column_pass_equals_inverse_multiply_forward(N, order):
    rng = np.random.default_rng(N + 7 * order)
    a = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    V = rng.standard_normal(N)
    P = factor(N, order)
    # plain plans first: the stages alone reproduce numpy's transforms
    c, NS = a.copy(), 1
    for R in P:
        c = stage(c, N, R, NS, -1)
        NS *= R
    assert np.abs(c - np.fft.fft(a)).max() < 1e-12 * np.abs(c).max()
    # the fused schedule
    b, NS = a.copy(), 1
    for R in P[:-1]:
        b = stage(b, N, R, NS, +1)
        NS *= R
    b = fused(b, N, P[-1], V)
    NS = P[-1]
    for R in P[::-1][1:]:
        b = stage(b, N, R, NS, -1)
        NS *= R
    want = np.fft.fft(V * np.fft.ifft(a) * N)
    assert np.abs(b - want).max() < 1e-12 * np.abs(want).max()
