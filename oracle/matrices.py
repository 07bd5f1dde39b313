"""Explicit unitary matrices and partial sensing matrices (FP64).

Sec. I: Phi = S_Omega A, with S_Omega the M x N row selector of the index set
Omega.  Sec. I lists two constraints on U (unimodular entries of magnitude
1/sqrt(N); columns of sqrt(N) U closed under elementwise product) that hold
for the two matrices built here.

Conventions (0-based indices; the paper is 1-based):
* Hadamard: the Sylvester construction H_1 = [1], H_{2n} = [[H, H], [H, -H]],
  scaled by 1/sqrt(N).  Built by repeated Kronecker products, not from a
  closed form, so that tests can pin the closed form against it.
* Fourier: A(i, k) = exp(-2 pi i i k / N) / sqrt(N).
"""
from __future__ import annotations

import numpy as np


def hadamard(N: int) -> np.ndarray:
    """Unitary Sylvester Hadamard matrix of order N = 2^n (FP64)."""
    if N < 1 or N & (N - 1):
        raise ValueError("N must be a power of two")
    H = np.ones((1, 1))
    h2 = np.array([[1.0, 1.0], [1.0, -1.0]])
    while H.shape[0] < N:
        H = np.kron(h2, H)
    return H / np.sqrt(N)


def fourier(N: int) -> np.ndarray:
    """Unitary DFT matrix, A(i,k) = exp(-2 pi i ik/N)/sqrt(N) (complex128)."""
    i = np.arange(N, dtype=np.int64)
    ph = np.outer(i, i) % N
    return np.exp(-2j * np.pi * ph / N) / np.sqrt(N)


def unitary(kind: str, N: int) -> np.ndarray:
    if kind == "wht":
        return hadamard(N)
    if kind == "dft":
        return fourier(N)
    raise ValueError(f"unknown kind {kind!r}")


def row_selector(N: int, omega) -> np.ndarray:
    """S_Omega: the M x N matrix made of rows Omega of the identity (Sec. I)."""
    S = np.zeros((len(omega), N))
    S[np.arange(len(omega)), np.asarray(omega, dtype=np.int64)] = 1.0
    return S


def sensing(kind: str, N: int, omega) -> np.ndarray:
    """Phi = S_Omega A (Sec. I), as a dense M x N array."""
    return row_selector(N, omega) @ unitary(kind, N)


def sensing_rows(kind: str, N: int, omega) -> np.ndarray:
    """Phi = S_Omega A built row by row from the entries of A, for N too large
    to form A itself: A(i,k) = (-1)^popcount(i&k)/sqrt(N) (Sylvester; pinned
    against the Kronecker construction in the tests) or
    exp(-2 pi i (ik mod N)/N)/sqrt(N)."""
    om = np.asarray(omega, dtype=np.int64)[:, None]
    k = np.arange(N, dtype=np.int64)[None, :]
    if kind == "wht":
        return (1.0 - 2.0 * (np.bitwise_count(om & k) & 1)) / np.sqrt(N)
    return np.exp(-2j * np.pi * ((om * k) % N) / N) / np.sqrt(N)
