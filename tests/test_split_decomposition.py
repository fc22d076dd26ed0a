"""The split passes' decomposition of the column transform, checked against numpy's FFT on the
CPU (no GPU, no library): for N = Q L, decimation in frequency over the rows,
n = n1 + L n2, k = Q k1 + k2,

    y[n1][k2] = W_N^{n1 k2} sum_{n2} x[n1 + L n2] W_Q^{n2 k2},   X[Q k1 + k2] = sum_{n1} y[n1][k2] W_L^{n1 k1},

with chunk k2 of the buffer holding y[.][k2] at rows k2 L + n1 (after its L-point transform,
X[Q k1 + k2] at row k2 L + k1), and the inverse the conjugate sums in the reverse order.  The
same index map gives the permuted copy of the modulus (row k2 L + k1 of it = row Q k1 + k2 of
M), so a pointwise step in the chunked layout is the pointwise step in natural order.  These
are the sides and radices of the split passes: Q = 3 at 192, 384, 768; 2 at 512; 8 at 1024."""
import numpy as np
import pytest

SPLIT = {192: 3, 384: 3, 512: 2, 768: 3, 1024: 8}


def first_stage(x, Q, sign):
    """Radix-Q stage over the rows of x (N x C) with twiddles W_N^{sign n1 k2}: the chunked
    layout (chunk k2 at rows k2 L + n1).  sign = -1 forward, +1 inverse (unnormalised)."""
    N = x.shape[0]
    L = N // Q
    n1 = np.arange(L)[:, None]
    out = np.empty_like(x)
    for k2 in range(Q):
        acc = sum(x[n1[:, 0] + L * n2] * np.exp(sign * 2j * np.pi * n2 * k2 / Q) for n2 in range(Q))
        out[k2 * L:(k2 + 1) * L] = acc * np.exp(sign * 2j * np.pi * n1 * k2 / N)
    return out


def chunk_ffts(y, Q, inverse=False):
    N = y.shape[0]
    L = N // Q
    f = (lambda a: np.fft.ifft(a, axis=0) * L) if inverse else (lambda a: np.fft.fft(a, axis=0))
    return np.concatenate([f(y[k2 * L:(k2 + 1) * L]) for k2 in range(Q)])


def chunk_order(N, Q):
    """Row k2 L + k1 of the chunked layout holds natural row Q k1 + k2."""
    L = N // Q
    return np.array([Q * k1 + k2 for k2 in range(Q) for k1 in range(L)])


@pytest.mark.parametrize("N", sorted(SPLIT))
def test_forward_split_equals_the_column_transform(N):
    Q = SPLIT[N]
    rng = np.random.default_rng(N)
    x = rng.standard_normal((N, 5)) + 1j * rng.standard_normal((N, 5))
    X = np.fft.fft(x, axis=0)
    Y = chunk_ffts(first_stage(x, Q, -1), Q)
    assert np.allclose(Y, X[chunk_order(N, Q)], rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("N", sorted(SPLIT))
def test_inverse_split_equals_the_unnormalised_inverse(N):
    Q = SPLIT[N]
    rng = np.random.default_rng(N + 1)
    X = rng.standard_normal((N, 4)) + 1j * rng.standard_normal((N, 4))
    Ychunked = X[chunk_order(N, Q)]
    # inverse: the L-point inverse of each chunk, then the inverse first stage
    x = first_stage_inverse(chunk_ffts(Ychunked, Q, inverse=True), Q)
    assert np.allclose(x, np.fft.ifft(X, axis=0) * N, rtol=1e-12, atol=1e-9)


def first_stage_inverse(y, Q):
    """x[n1 + L n2] = sum_{k2} W_Q^{-n2 k2} W_N^{-n1 k2} y[n1][k2] (chunk k2 at rows k2 L + n1)."""
    N = y.shape[0]
    L = N // Q
    n1 = np.arange(L)[:, None]
    out = np.empty_like(y)
    for n2 in range(Q):
        out[n2 * L:(n2 + 1) * L] = sum(
            y[k2 * L:(k2 + 1) * L] * np.exp(2j * np.pi * n1 * k2 / N) * np.exp(2j * np.pi * n2 * k2 / Q)
            for k2 in range(Q))
    # out is in row order n2 L + n1 = natural row n1 + L n2
    return out


@pytest.mark.parametrize("N", sorted(SPLIT))
def test_pointwise_step_in_the_chunked_layout(N):
    # a modulus projection applied in the chunked layout with the permuted modulus equals the
    # projection in natural order: the whole split iteration is the plain one, reordered
    Q = SPLIT[N]
    rng = np.random.default_rng(N + 2)
    x = rng.standard_normal((N, 3)) + 1j * rng.standard_normal((N, 3))
    M = rng.uniform(0.1, 2.0, (N, 3))
    X = np.fft.fft(x, axis=0)
    ref = np.fft.ifft(M * X / np.abs(X), axis=0) * N
    Y = chunk_ffts(first_stage(x, Q, -1), Q)
    Mp = M[chunk_order(N, Q)]
    got = first_stage_inverse(chunk_ffts(Mp * Y / np.abs(Y), Q, inverse=True), Q)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-9)


def test_split_sides_have_power_of_two_chunks():
    # the chunks the column pass transforms are powers of two at every split side
    for N, Q in SPLIT.items():
        L = N // Q
        assert N == Q * L and L & (L - 1) == 0
