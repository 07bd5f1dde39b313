"""Algorithm 1.1 (conventional OMP), dense FP64.

Steps as numbered in Algorithm 1.1 (Sec. I):
 1) r_0 = y, Lambda_0 = {}, t = 1
 2) h_{t-1} = Phi^H r_{t-1}                     (dense matrix-vector product)
 3) lambda_t = argmax_j |h_{t-1}(j)|
 4) Lambda_t = Lambda_{t-1} + {lambda_t}
 5) Phi_t = Phi S_{Lambda_t}^T
 6) x_t = (Phi_t^H Phi_t)^{-1} Phi_t^H y        (normal equations, Cholesky)
 7) a_t = Phi_t x_t, r_t = y - a_t
 8) t = t + 1, back to 2) unless halted

Readings where the paper is silent (stated identically for the GPU path):
* identification compares |h(j)|^2, skips indices already in Lambda, and
  breaks ties by the smallest j;
* halting after step 7): stop when t = K or ||r_t|| < rel_tol ||y||;
* a zero measurement (||y|| = 0) halts before the first iteration;
* a selected column whose Cholesky pivot d^2 = G_tt - ||L^{-1} g||^2 is at or
  below ``dep_tol * (M/N)`` is numerically dependent on Lambda: the run stops
  without adding it.
"""
from __future__ import annotations

import numpy as np

DEP_TOL = 1e-10


def correlate(Phi: np.ndarray, r: np.ndarray) -> np.ndarray:
    """Step 2): h = Phi^H r (dense)."""
    return Phi.conj().T @ r


def identify(h: np.ndarray, excluded) -> tuple[int, float]:
    """Step 3): index of the largest |h(j)|^2 outside ``excluded``, lowest j on
    ties, plus the relative gap (|h|_(1) - |h|_(2)) / |h|_(1) between the two
    largest magnitudes (1.0 when fewer than two candidates or h = 0)."""
    score = (h.conj() * h).real.astype(np.float64)
    score = score.copy()
    if len(excluded):
        score[np.asarray(excluded, dtype=np.int64)] = -np.inf
    j = int(np.argmax(score))  # first maximum = lowest index
    s = score.copy()
    s[j] = -np.inf
    top1 = np.sqrt(max(score[j], 0.0))
    top2 = np.sqrt(max(np.max(s), 0.0)) if np.isfinite(np.max(s)) else 0.0
    gap = 1.0 if top1 == 0.0 else (top1 - top2) / top1
    return j, float(gap)


def least_squares(Phi_t: np.ndarray, y: np.ndarray) -> tuple[np.ndarray, float]:
    """Step 6): x = (Phi_t^H Phi_t)^{-1} Phi_t^H y by a Cholesky factor of the
    explicitly formed Gram matrix.  Returns x and the last pivot d^2."""
    G = Phi_t.conj().T @ Phi_t
    b = Phi_t.conj().T @ y
    L = np.linalg.cholesky(G)
    # last pivot, recomputed from the factor of the leading block
    t = G.shape[0]
    if t == 1:
        d2 = float(G[0, 0].real)
    else:
        w = np.linalg.solve(L[: t - 1, : t - 1], G[: t - 1, t - 1])
        d2 = float((G[t - 1, t - 1] - np.vdot(w, w)).real)
    z = np.linalg.solve(L, b)
    x = np.linalg.solve(L.conj().T, z)
    return x, d2


def omp(Phi: np.ndarray, y: np.ndarray, K: int, rel_tol: float = 1e-6, dep_tol: float = DEP_TOL,
        record_h: bool = False) -> dict:
    """Run Algorithm 1.1 for at most K iterations.

    Returns support (selection order), x (on the support), iters, resnorm
    history ||r_t||, the identification gap of every iteration and, with
    ``record_h``, every correlation vector h_{t-1}.
    """
    M, N = Phi.shape
    y = np.asarray(y).astype(np.complex128 if np.iscomplexobj(Phi) or np.iscomplexobj(y) else np.float64)
    ynorm = float(np.linalg.norm(y))
    out = {"support": [], "x": np.zeros(0, dtype=y.dtype), "iters": 0, "resnorm": [],
           "gap": [], "h": [], "d2": [], "halt": "max_iter", "ynorm": ynorm}
    if ynorm == 0.0 or K <= 0:
        out["halt"] = "zero_y" if ynorm == 0.0 else "max_iter"
        return out
    r = y.copy()                      # step 1
    lam: list[int] = []
    x = out["x"]
    for t in range(1, K + 1):
        h = correlate(Phi, r)         # step 2
        if record_h:
            out["h"].append(h)
        j, gap = identify(h, lam)     # step 3
        trial = lam + [j]             # step 4
        Phi_t = Phi[:, trial]         # step 5
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
        x, _ = least_squares(Phi_t, y)  # step 6
        r = y - Phi_t @ x             # step 7
        rn = float(np.linalg.norm(r))
        out["resnorm"].append(rn)
        if rn < rel_tol * ynorm:
            out["halt"] = "tolerance"
            break
    out["support"] = lam
    out["x"] = x
    out["iters"] = len(lam)
    return out
