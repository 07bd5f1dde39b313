"""Algorithm 1.1 for large N, FP64, with the correlation of step 2 and the
residual of step 7 computed by transforms instead of a dense Phi.

Test infrastructure only.  For N of 2^14 and more a dense M x N Phi no
longer fits in memory, so this variant applies Phi and Phi^H through the
unitary transform A (Sec. I: Phi = S_Omega A):

  Phi^H r = A^H zf_Omega(r),        Phi x_Lambda = (A zf_Lambda(x))(Omega),

with A^H v = sqrt(N) * ifft(v) and A v = fft(v) / sqrt(N) for the Fourier
matrix A(i, k) = exp(-2 pi i ik/N)/sqrt(N) (numpy's FFT as a library
primitive), and A v = A^H v = fwht(v) / sqrt(N) for the Sylvester Hadamard
matrix, fwht being the radix-2 butterflies written out below.  The least
squares of step 6 forms Phi_t from the closed-form entries of its columns and
calls the dense oracle's Cholesky solve; identification and halting are the
dense oracle's (oracle.omp), so the two differ only in how Phi is applied.
Subspace pursuit and CoSaMP follow oracle.pursuits step for step with the
same substitution.  Tests pin this module against the dense oracle at
N <= 4096.
"""
from __future__ import annotations

import numpy as np

from .omp import DEP_TOL, identify, least_squares


def fwht(v: np.ndarray) -> np.ndarray:
    """Unnormalised Sylvester Walsh-Hadamard transform along the last axis:
    log2 N stages of butterflies (a, b) -> (a + b, a - b) on pairs h apart."""
    a = np.array(v, dtype=np.result_type(v, np.float64), copy=True)
    N = a.shape[-1]
    if N & (N - 1):
        raise ValueError("length must be a power of two")
    lead = a.shape[:-1]
    h = 1
    while h < N:
        a = a.reshape(*lead, N // (2 * h), 2, h)
        top, bot = a[..., 0, :], a[..., 1, :]
        a = np.stack((top + bot, top - bot), axis=-2)
        h *= 2
    return a.reshape(*lead, N)


def apply_A(kind: str, v: np.ndarray) -> np.ndarray:
    """A v for the unitary A of the kind (last axis)."""
    N = v.shape[-1]
    if kind == "dft":
        return np.fft.fft(v, axis=-1) / np.sqrt(N)
    return fwht(v) / np.sqrt(N)


def apply_AH(kind: str, v: np.ndarray) -> np.ndarray:
    """A^H v for the unitary A of the kind (last axis)."""
    N = v.shape[-1]
    if kind == "dft":
        return np.fft.ifft(v, axis=-1) * np.sqrt(N)
    return fwht(v) / np.sqrt(N)


def zero_fill(N: int, idx, vals) -> np.ndarray:
    """zf(v): the length-N vector with vals at idx and 0 elsewhere."""
    vals = np.asarray(vals)
    out = np.zeros(N, dtype=np.result_type(vals, np.float64))
    out[np.asarray(idx, dtype=np.int64)] = vals
    return out


def correlate(kind: str, N: int, omega, r) -> np.ndarray:
    """Step 2): h = Phi^H r = A^H zf_Omega(r)."""
    return apply_AH(kind, zero_fill(N, omega, r))


def synthesize(kind: str, N: int, omega, support, x) -> np.ndarray:
    """Phi_Lambda x = (A zf_Lambda(x))(Omega)."""
    return apply_A(kind, zero_fill(N, support, x))[np.asarray(omega, dtype=np.int64)]


def kernel_vector(kind: str, N: int, omega) -> np.ndarray:
    """c = U^H S^T S U e_0 (Eq. kernelsum): U e_0 is the constant column
    1/sqrt(N), so c = A^H zf_Omega(1) / sqrt(N)."""
    return correlate(kind, N, omega, np.ones(len(omega))) / np.sqrt(N)


def columns(kind: str, N: int, omega, support) -> np.ndarray:
    """Phi[:, support] from the closed-form entries of A (M x s)."""
    om = np.asarray(omega, dtype=np.int64)[:, None]
    k = np.asarray(support, dtype=np.int64)[None, :]
    if kind == "wht":
        return (1.0 - 2.0 * (np.bitwise_count(om & k) & 1)) / np.sqrt(N)
    return np.exp(-2j * np.pi * ((om * k) % N) / N) / np.sqrt(N)


def omp(kind: str, N: int, omega, y, K: int, rel_tol: float = 1e-6, dep_tol: float = DEP_TOL,
        record_x: bool = False) -> dict:
    """Algorithm 1.1 with transform-based steps 2 and 7; same outputs as
    oracle.omp.omp (support in selection order, x, iters, resnorm history,
    gaps, d2, halt); with ``record_x`` also every iterate x_t ("xs")."""
    omega = np.asarray(omega, dtype=np.int64)
    M = len(omega)
    cplx = kind == "dft" or np.iscomplexobj(y)
    y = np.asarray(y).astype(np.complex128 if cplx else np.float64)
    ynorm = float(np.linalg.norm(y))
    out = {"support": [], "x": np.zeros(0, dtype=y.dtype), "iters": 0, "resnorm": [],
           "gap": [], "d2": [], "halt": "max_iter", "ynorm": ynorm}
    if ynorm == 0.0 or K <= 0:
        out["halt"] = "zero_y" if ynorm == 0.0 else "max_iter"
        return out
    r = y.copy()                                   # step 1
    lam: list[int] = []
    x = out["x"]
    for t in range(1, K + 1):
        h = correlate(kind, N, omega, r)           # step 2
        j, gap = identify(h, lam)                  # step 3
        trial = lam + [j]                          # step 4
        Phi_t = columns(kind, N, omega, trial)     # step 5
        G = Phi_t.conj().T @ Phi_t
        if t > 1:
            L = np.linalg.cholesky(G[: t - 1, : t - 1])
            w = np.linalg.solve(L, G[: t - 1, t - 1])
            d2 = float((G[t - 1, t - 1] - np.vdot(w, w)).real)
        else:
            d2 = float(G[0, 0].real)
        if d2 <= dep_tol * (M / N):
            out["halt"] = "dependent"
            break
        lam = trial
        out["gap"].append(gap)
        out["d2"].append(d2)
        x, _ = least_squares(Phi_t, y)             # step 6
        if record_x:
            out.setdefault("xs", []).append(x)
        r = y - synthesize(kind, N, omega, lam, x)  # step 7
        rn = float(np.linalg.norm(r))
        out["resnorm"].append(rn)
        if rn < rel_tol * ynorm:
            out["halt"] = "tolerance"
            break
    out["support"] = lam
    out["x"] = x
    out["iters"] = len(lam)
    return out


def _ls_cols(kind, N, omega, y, cols):
    """Least squares on the columns `cols` (the dense oracle's Cholesky solve on
    the closed-form columns)."""
    from .pursuits import ls
    cols = np.asarray(cols, dtype=np.int64)
    if len(cols) == 0:
        return np.zeros(0, dtype=y.dtype)
    return ls(columns(kind, N, omega, cols), y, np.arange(len(cols)))


def subspace_pursuit(kind: str, N: int, omega, y, K: int, max_iter: int | None = None,
                     rel_tol: float = 1e-6) -> dict:
    """oracle.pursuits.subspace_pursuit with Phi applied through transforms
    (same steps, same readings), for N too large for a dense Phi."""
    from .pursuits import top_k
    omega = np.asarray(omega, dtype=np.int64)
    y = np.asarray(y).astype(np.complex128 if kind == "dft" or np.iscomplexobj(y) else np.float64)
    ynorm = float(np.linalg.norm(y))
    max_iter = K if max_iter is None else max_iter
    out = {"support": np.zeros(0, np.int64), "x": np.zeros(0, y.dtype), "iters": 0, "resnorm": [ynorm],
           "ynorm": ynorm}
    if ynorm == 0.0 or K <= 0:
        return out
    res = lambda cols, x: y - synthesize(kind, N, omega, cols, x) if len(cols) else y
    T = top_k(correlate(kind, N, omega, y), K)
    x = _ls_cols(kind, N, omega, y, T)
    rn = float(np.linalg.norm(res(T, x)))
    out["resnorm"] = [rn]
    it = 0
    while it < max_iter and rn >= rel_tol * ynorm:
        h = correlate(kind, N, omega, res(T, x))
        Tp = np.union1d(T, top_k(h, K, excluded=T))
        b = _ls_cols(kind, N, omega, y, Tp)
        Tn = np.sort(Tp[top_k(b, K)])
        xn = _ls_cols(kind, N, omega, y, Tn)
        rn_new = float(np.linalg.norm(res(Tn, xn)))
        it += 1
        if rn_new >= rn:
            break
        T, x, rn = Tn, xn, rn_new
        out["resnorm"].append(rn)
    out.update(support=T, x=x, iters=it)
    return out


def cosamp(kind: str, N: int, omega, y, K: int, max_iter: int = 50, rel_tol: float = 1e-6) -> dict:
    """oracle.pursuits.cosamp with Phi applied through transforms."""
    from .pursuits import top_k
    omega = np.asarray(omega, dtype=np.int64)
    y = np.asarray(y).astype(np.complex128 if kind == "dft" or np.iscomplexobj(y) else np.float64)
    ynorm = float(np.linalg.norm(y))
    out = {"support": np.zeros(0, np.int64), "x": np.zeros(0, y.dtype), "iters": 0, "resnorm": [ynorm],
           "ynorm": ynorm}
    if ynorm == 0.0 or K <= 0:
        return out
    res = lambda cols, x: y - synthesize(kind, N, omega, cols, x) if len(cols) else y
    S = np.zeros(0, np.int64)
    x = np.zeros(0, y.dtype)
    rn = ynorm
    it = 0
    while it < max_iter and rn >= rel_tol * ynorm:
        h = correlate(kind, N, omega, res(S, x))
        T = np.union1d(top_k(h, 2 * K), S)
        b = _ls_cols(kind, N, omega, y, T)
        keep = top_k(b, K)
        Sn, xn = T[keep], b[keep]
        rn_new = float(np.linalg.norm(res(Sn, xn)))
        it += 1
        if rn_new >= rn:
            break
        S, x, rn = Sn, xn, rn_new
        out["resnorm"].append(rn)
    out.update(support=S, x=x, iters=it)
    return out
