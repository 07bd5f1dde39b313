"""Subspace pursuit (SP) and CoSaMP, dense FP64.

The paper applies its fast correlation to "almost all MPAs" (Sec. I) and
reports the cost of a fast CoSaMP (Sec. IV, Fig. 3) but describes neither
algorithm.  These are their standard forms (SP: Dai and Milenkovic; CoSaMP:
Needell and Tropp), written with the same building blocks as Algorithm 1.1:
the correlation h = Phi^H r (step 2), least squares on a column set by the
normal equations (step 6) and the residual (step 7).

Readings (stated identically for the GPU path):
* top_k(v, k, excluded) returns the k indices with the largest |v(j)|^2 among
  j not excluded, ties to the lower index, as a sorted array;
* SP: T_0 = top_K(Phi^H y), x = LS on T, r = y - Phi_T x.  Each iteration:
  T' = T + top_K(Phi^H r) over j not in T; b = LS on T'; T_new = the K
  entries of b with the largest |b|; x_new = LS on T_new; stop, keeping the
  previous iterate, when ||r_new|| >= ||r||; otherwise accept, and stop when
  ||r|| < rel_tol ||y|| or after max_iter iterations;
* CoSaMP: x = 0, r = y.  Each iteration: T = top_2K(Phi^H r) (all j) joined
  with supp(x); b = LS on T; x_new = b kept on its K largest |b| (no second
  solve); stop, keeping the previous iterate, when ||r_new|| >= ||r||;
  otherwise accept, and stop when ||r|| < rel_tol ||y|| or after max_iter;
* a zero measurement returns x = 0 with no iteration.

Each run returns a trace of its iterations (SP: T', b, T_new, x_new and
||r_new|| with the acceptance; CoSaMP: T, b, the kept set, x_new and ||r_new||
with the acceptance).  The paper prints no iterate; the pins are iterates
derived by hand for tiny cases (exact in binary arithmetic or with clear gaps
between the k-th and (k+1)-th magnitudes), recovery, and the invariants each
step defines (tests/test_oracle_pursuits.py).
"""
from __future__ import annotations

import numpy as np


def top_k(v: np.ndarray, k: int, excluded=()) -> np.ndarray:
    """Indices of the k largest |v(j)|^2 over j not in `excluded`, lowest j
    first among equal values; returned sorted ascending."""
    score = (np.conj(v) * v).real.astype(np.float64).copy()
    if len(excluded):
        score[np.asarray(list(excluded), dtype=np.int64)] = -np.inf
    order = np.lexsort((np.arange(len(score)), -score))  # by -score, then index
    sel = [int(j) for j in order[:k] if np.isfinite(score[j])]
    return np.array(sorted(sel), dtype=np.int64)


def ls(Phi: np.ndarray, y: np.ndarray, cols) -> np.ndarray:
    """x = (Phi_T^H Phi_T)^{-1} Phi_T^H y by a Cholesky factor (step 6)."""
    cols = np.asarray(cols, dtype=np.int64)
    if len(cols) == 0:
        return np.zeros(0, dtype=y.dtype)
    P = Phi[:, cols]
    G = P.conj().T @ P
    L = np.linalg.cholesky(G)
    z = np.linalg.solve(L, P.conj().T @ y)
    return np.linalg.solve(L.conj().T, z)


def _residual(Phi, y, cols, x):
    cols = np.asarray(cols, dtype=np.int64)
    return y - (Phi[:, cols] @ x if len(cols) else 0.0)


def subspace_pursuit(Phi: np.ndarray, y: np.ndarray, K: int, max_iter: int | None = None,
                     rel_tol: float = 1e-6) -> dict:
    M, N = Phi.shape
    y = np.asarray(y).astype(np.complex128 if np.iscomplexobj(Phi) or np.iscomplexobj(y) else np.float64)
    ynorm = float(np.linalg.norm(y))
    max_iter = K if max_iter is None else max_iter
    out = {"support": np.zeros(0, np.int64), "x": np.zeros(0, y.dtype), "iters": 0, "resnorm": [ynorm],
           "ynorm": ynorm}
    if ynorm == 0.0 or K <= 0:
        return out
    T = top_k(Phi.conj().T @ y, K)
    x = ls(Phi, y, T)
    rn = float(np.linalg.norm(_residual(Phi, y, T, x)))
    out["resnorm"] = [rn]
    out["T0"], out["x0"], out["trace"] = T, x, []
    it = 0
    while it < max_iter and rn >= rel_tol * ynorm:
        r = _residual(Phi, y, T, x)
        h = Phi.conj().T @ r
        Tp = np.union1d(T, top_k(h, K, excluded=T))
        b = ls(Phi, y, Tp)
        Tn = np.sort(Tp[top_k(b, K)])
        xn = ls(Phi, y, Tn)
        rn_new = float(np.linalg.norm(_residual(Phi, y, Tn, xn)))
        it += 1
        out["trace"].append({"Tp": Tp, "b": b, "Tn": Tn, "x": xn, "rn": rn_new, "accepted": rn_new < rn})
        if rn_new >= rn:
            break
        T, x, rn = Tn, xn, rn_new
        out["resnorm"].append(rn)
    out.update(support=T, x=x, iters=it)
    return out


def cosamp(Phi: np.ndarray, y: np.ndarray, K: int, max_iter: int = 50, rel_tol: float = 1e-6) -> dict:
    M, N = Phi.shape
    y = np.asarray(y).astype(np.complex128 if np.iscomplexobj(Phi) or np.iscomplexobj(y) else np.float64)
    ynorm = float(np.linalg.norm(y))
    out = {"support": np.zeros(0, np.int64), "x": np.zeros(0, y.dtype), "iters": 0, "resnorm": [ynorm],
           "ynorm": ynorm}
    if ynorm == 0.0 or K <= 0:
        return out
    S = np.zeros(0, np.int64)
    x = np.zeros(0, y.dtype)
    rn = ynorm
    out["trace"] = []
    it = 0
    while it < max_iter and rn >= rel_tol * ynorm:
        r = _residual(Phi, y, S, x)
        h = Phi.conj().T @ r
        T = np.union1d(top_k(h, 2 * K), S)
        b = ls(Phi, y, T)
        keep = top_k(b, K)
        Sn, xn = T[keep], b[keep]
        rn_new = float(np.linalg.norm(_residual(Phi, y, Sn, xn)))
        it += 1
        out["trace"].append({"T": T, "b": b, "S": Sn, "x": xn, "rn": rn_new, "accepted": rn_new < rn})
        if rn_new >= rn:
            break
        S, x, rn = Sn, xn, rn_new
        out["resnorm"].append(rn)
    out.update(support=S, x=x, iters=it)
    return out
