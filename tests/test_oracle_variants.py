"""Pins behind the paper's storage variants and deterministic row sets
(Sec. I, Sec. III-B), CPU only: the DFT kernel vector is conjugate symmetric
for every Omega (half storage is lossless), N c is an integer for the WHT (the
integer storage is exact), and two deterministic Omega have closed-form
kernel vectors that the oracle reproduces."""
import numpy as np
import pytest

import synth
from oracle import kernelsum, transform as tro


@pytest.mark.parametrize("N,M", [(16, 5), (1024, 300), (8192, 2048)])
def test_dft_kernel_vector_conjugate_symmetric(N, M):
    om = synth.draw_omega(N, M, np.random.default_rng(N))
    c = tro.kernel_vector("dft", N, om)
    d = np.arange(N)
    assert np.max(np.abs(c[(-d) % N] - np.conj(c))) < 1e-15


@pytest.mark.parametrize("N,M", [(16, 5), (1024, 300), (1 << 14, 4000)])
def test_wht_kernel_vector_integer_counts(N, M):
    om = synth.draw_omega(N, M, np.random.default_rng(N + 1))
    c = tro.kernel_vector("wht", N, om)
    # N c(d) = M - 2 #{i in Omega : popcount(i & d) odd}, counted directly
    d = np.arange(N, dtype=np.int64)[:, None] if N <= 1024 else np.arange(0, N, 97, dtype=np.int64)[:, None]
    odd = (np.bitwise_count(om.astype(np.int64)[None, :] & d) & 1).astype(np.int64).sum(axis=1)
    want = M - 2 * odd
    got = N * c[d[:, 0]]
    assert np.array_equal(np.round(got), want) and np.max(np.abs(got - want)) < 1e-9


@pytest.mark.parametrize("N,M", [(64, 16), (4096, 1000)])
def test_contiguous_omega_dirichlet_kernel(N, M):
    """Omega = {0, ..., M-1} (a low-pass row set): c(d) = (1/N) sum_{i<M}
    e^{2 pi i id/N}, a geometric sum with closed form
    e^{i pi (M-1) d/N} sin(pi M d/N) / (N sin(pi d/N)), c(0) = M/N."""
    om = np.arange(M, dtype=np.int32)
    c = tro.kernel_vector("dft", N, om)
    d = np.arange(1, N)
    want = np.exp(1j * np.pi * (M - 1) * d / N) * np.sin(np.pi * M * d / N) / (N * np.sin(np.pi * d / N))
    assert abs(c[0] - M / N) < 1e-15
    assert np.max(np.abs(c[1:] - want)) < 1e-13
    assert np.max(np.abs(kernelsum.kernel_vector("dft", N, om) - c)) < 1e-13 if N <= 64 else True


def test_subspace_omega_wht_kernel_is_indicator_of_dual():
    """Omega = a linear subspace of F_2^n (the rows of a code's codewords):
    c(d) = M/N if d is orthogonal to every element of Omega, else 0."""
    n, basis = 10, [0b0000000011, 0b0000111100, 0b1101000000, 0b0010010001]
    span = {0}
    for v in basis:
        span |= {s ^ v for s in span}
    om = np.array(sorted(span), dtype=np.int32)
    N, M = 1 << n, len(om)
    c = tro.kernel_vector("wht", N, om)
    dual = np.array([all(bin(d & v).count("1") % 2 == 0 for v in basis) for d in range(N)])
    assert np.max(np.abs(c - np.where(dual, M / N, 0.0))) < 1e-15
    assert dual.sum() == N // M
