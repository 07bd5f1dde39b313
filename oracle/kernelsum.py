"""Correlation kernel vector and the fast correlation of Sec. II-III (FP64).

* Eq. (kernelsum): c = U^H S_Omega^T S_Omega U e_1, the correlation kernel
  vector (e_1 is the first column of I; 0-based here: e_0).
* Theorem 2-1: P_lambda = U^H D_lambda U with D_lambda = sqrt(N) diag(u_lambda)
  is a permutation matrix.
* Eq. (kernelsum) / (kernelsumOMP):
      h_t = h_0 - sum_tau x_t(tau) P_{Lambda_t(tau)} c,  h_0 = U^H S_Omega^T y.

``fast_correlation_dense`` evaluates that sum with the dense P_lambda of the
theorem's definition.  ``fast_correlation`` applies P_lambda as the index map
the paper names for each matrix (Sec. III-B: a cyclic shift for the Fourier
matrix; compositions of the log2 N bit-flip permutations for the Hadamard
matrix), i.e. (P_lambda c)(j) = c((j - lambda) mod N) or c(j XOR lambda).  A
test pins the index map against the dense P_lambda.
"""
from __future__ import annotations

import numpy as np

from .matrices import row_selector, unitary


def kernel_vector(kind: str, N: int, omega) -> np.ndarray:
    """c = U^H S^T S U e_0 (Eq. kernelsum), straight from the definition."""
    U = unitary(kind, N)
    S = row_selector(N, omega)
    e0 = np.zeros(N)
    e0[0] = 1.0
    return U.conj().T @ (S.T @ (S @ (U @ e0)))


def kernel_vector_rows(kind: str, N: int, omega) -> np.ndarray:
    """c(j) = sum_{i in Omega} conj(U(i, j)) U(i, 0): Eq. (kernelsum) expanded
    entry by entry over the rows of Phi, for N too large for a dense U."""
    from .matrices import sensing_rows
    Phi = sensing_rows(kind, N, omega)
    return Phi.conj().T @ Phi[:, 0] if len(Phi) else np.zeros(N)


def permutation(kind: str, N: int, lam: int) -> np.ndarray:
    """P_lambda = U^H D_lambda U, D_lambda = sqrt(N) diag(u_lambda) (Theorem 2-1)."""
    U = unitary(kind, N)
    D = np.sqrt(N) * np.diag(U[:, lam])
    return U.conj().T @ D @ U


def initial_correlation(kind: str, N: int, omega, y) -> np.ndarray:
    """h_0 = U^H S_Omega^T y (Eq. corr_com)."""
    U = unitary(kind, N)
    S = row_selector(N, omega)
    return U.conj().T @ (S.T @ np.asarray(y))


def shift_index(kind: str, N: int, j, lam: int):
    """Row j of P_lambda has its single 1 in column shift_index(j, lambda)."""
    j = np.asarray(j, dtype=np.int64)
    if kind == "dft":
        return (j - lam) % N
    return j ^ lam


def fast_correlation_dense(kind: str, N: int, c, h0, support, x) -> np.ndarray:
    """h = h_0 - sum_tau x(tau) P_{support(tau)} c with dense P (Eq. kernelsum)."""
    h = np.array(h0, dtype=np.complex128 if kind == "dft" else np.float64)
    for lam, xv in zip(support, x):
        h = h - xv * (permutation(kind, N, int(lam)) @ c)
    return h


def fast_correlation(kind: str, N: int, c, h0, support, x) -> np.ndarray:
    """h(j) = h_0(j) - sum_tau x(tau) c(j (-) support(tau)) (Eq. kernelsumOMP)."""
    h = np.array(h0, dtype=np.complex128 if kind == "dft" else np.float64)
    j = np.arange(N)
    c = np.asarray(c)
    for lam, xv in zip(support, x):
        h = h - xv * c[shift_index(kind, N, j, int(lam))]
    return h


def gram_from_kernel(kind: str, N: int, c, support) -> np.ndarray:
    """G(a, b) = (Phi_Lambda^H Phi_Lambda)(a, b) = c(Lambda_a (-) Lambda_b).

    Row Lambda_a of P_{Lambda_b} c, i.e. the Gram entries read off c."""
    s = np.asarray(support, dtype=np.int64)
    c = np.asarray(c)
    return c[shift_index(kind, N, s[:, None], s[None, :])]
