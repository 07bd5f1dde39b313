"""Seeded synthetic compressed-sensing instances (measurement model only).

This module draws the inputs that both the FP64 oracle and the CUDA path
consume: the row set Omega, the sparse signal x and the measurement
y = Phi x + eta of the problem statement (Sec. I, Eq. CSbasic).  It holds no
part of the recovery method: no correlation, no transform, no least squares.
The entries Phi(m, k) = A(Omega_m, k) it needs are evaluated from their closed
forms one column at a time (Sec. I: Phi = S_Omega A):

* WHT (Sylvester):  A(i, k) = (-1)^popcount(i & k) / sqrt(N)
* DFT:              A(i, k) = exp(-2 pi i * (i k mod N) / N) / sqrt(N)

Generation recipe (the paper fixes none of it; these are the stated readings):
Omega is drawn uniformly without replacement and sorted ascending; the support
is K distinct indices drawn uniformly; nonzeros are N(0,1) (real), CN(0,1)
(complex, re/im each N(0,1/2)) or Rademacher +-1; noise is added per instance
at the requested SNR, sigma^2 = ||Phi x||^2 / (M 10^(SNR/10)).  All draws use
numpy's PCG64 ``default_rng(seed)``.
"""
from __future__ import annotations

import functools

import numpy as np

WHT = "wht"
DFT = "dft"


def draw_omega(N: int, M: int, rng: np.random.Generator) -> np.ndarray:
    """M distinct row indices in [0, N), sorted ascending (int32)."""
    if not (0 <= M <= N):
        raise ValueError("need 0 <= M <= N")
    return np.sort(rng.choice(N, size=M, replace=False)).astype(np.int32)


def draw_support(N: int, K: int, rng: np.random.Generator) -> np.ndarray:
    """K distinct column indices in [0, N) in drawn order (int32)."""
    return rng.choice(N, size=K, replace=False).astype(np.int32)


def draw_values(K: int, kind: str, dist: str, rng: np.random.Generator) -> np.ndarray:
    """Nonzero values: 'gauss' (N(0,1) or CN(0,1)) or 'rademacher' (+-1)."""
    if dist == "gauss":
        if kind == DFT:
            return (rng.standard_normal(K) + 1j * rng.standard_normal(K)) / np.sqrt(2.0)
        return rng.standard_normal(K)
    if dist == "rademacher":
        s = rng.integers(0, 2, size=K) * 2.0 - 1.0
        return s.astype(np.complex128) if kind == DFT else s
    raise ValueError(f"unknown value distribution {dist!r}")


def sensing_column(kind: str, N: int, omega: np.ndarray, k: int) -> np.ndarray:
    """Column k of Phi = S_Omega A, from the closed form of A (FP64)."""
    om = omega.astype(np.int64)
    if kind == WHT:
        par = np.bitwise_count(om & np.int64(k)) & 1
        return (1.0 - 2.0 * par) / np.sqrt(N)
    ph = (om * np.int64(k)) % N
    return np.exp(-2j * np.pi * ph / N) / np.sqrt(N)


@functools.lru_cache(maxsize=8)
def _dft_entries(N: int) -> np.ndarray:
    """exp(-2 pi i p / N) / sqrt(N) for p = 0 .. N-1: the values the entries
    of A take (entry (i, k) is the one at p = i k mod N), each evaluated by
    the same expression as in sensing_column."""
    return np.exp(-2j * np.pi * np.arange(N, dtype=np.int64) / N) / np.sqrt(N)


def measure(kind: str, N: int, omega: np.ndarray, support: np.ndarray, values: np.ndarray) -> np.ndarray:
    """Noiseless y = Phi x for x supported on ``support`` (FP64 / complex128)."""
    y = np.zeros(len(omega), dtype=np.complex128 if kind == DFT else np.float64)
    if kind == DFT and len(support) > 8:
        # the same column values, looked up instead of re-evaluated per column
        om = omega.astype(np.int64)
        w = _dft_entries(N)
        for k, v in zip(support.tolist(), values.tolist()):
            y += v * w[(om * np.int64(k)) % N]
        return y
    for k, v in zip(support.tolist(), values.tolist()):
        y += v * sensing_column(kind, N, omega, k)
    return y


def add_noise(y: np.ndarray, snr_db: float | None, rng: np.random.Generator) -> np.ndarray:
    if snr_db is None:
        return y
    M = len(y)
    sigma2 = float(np.vdot(y, y).real) / (M * 10.0 ** (snr_db / 10.0))
    if np.iscomplexobj(y):
        eta = (rng.standard_normal(M) + 1j * rng.standard_normal(M)) * np.sqrt(sigma2 / 2.0)
    else:
        eta = rng.standard_normal(M) * np.sqrt(sigma2)
    return y + eta


def working_dtype(kind: str, prec: str):
    """numpy dtype of y / h in the given precision ('fp64' or 'fp32')."""
    if kind == DFT:
        return np.complex128 if prec == "fp64" else np.complex64
    return np.float64 if prec == "fp64" else np.float32


def make_batch(kind: str, N: int, M: int, K: int, B: int, *, snr_db=None, dist="gauss",
               prec="fp32", seed: int = 0, omega_seed: int | None = None) -> dict:
    """B instances sharing one Omega.

    Omega comes from ``default_rng(omega_seed)`` (``seed`` if None); instance b
    draws its support, values and noise from ``default_rng(seed + 1 + b)``.
    ``Y`` is stored in the working precision (rounded once); the oracle and
    the GPU both read that rounded array.
    """
    rng0 = np.random.default_rng(seed if omega_seed is None else omega_seed)
    omega = draw_omega(N, M, rng0)
    supports, values, ys = [], [], []
    for b in range(B):
        rng = np.random.default_rng(seed + 1 + b)
        s = draw_support(N, K, rng)
        v = draw_values(K, kind, dist, rng)
        y = add_noise(measure(kind, N, omega, s, v), snr_db, rng)
        supports.append(s)
        values.append(v)
        ys.append(y)
    dt = working_dtype(kind, prec)
    return {
        "kind": kind, "N": N, "M": M, "K": K, "B": B, "prec": prec,
        "omega": omega,
        "support": np.stack(supports) if B else np.zeros((0, K), np.int32),
        "values": np.stack(values) if B else np.zeros((0, K)),
        "Y": (np.stack(ys) if B else np.zeros((0, M))).astype(dt),
    }


# Workloads used by the tests and the benchmark (sizes, not data).
CONFIG_WHT_FP64_SINGLE = dict(kind=WHT, N=1024, M=256, K=16, B=1, snr_db=None, prec="fp64", seed=0)
CONFIG_DFT_C64_BATCH = dict(kind=DFT, N=4096, M=1024, K=64, B=1024, snr_db=40.0, prec="fp32", seed=0)


# Request stream of the serving workload: Poisson arrivals at `rate` per
# second; N = 2^e with e uniform over [log_n_lo, log_n_hi]; M = N / 8; K
# uniform over [k_lo, k_hi]; kind by a fair coin; OMP or CoSaMP by a fair
# coin, CoSaMP's K capped at M/3 (its least squares run on up to 3K of the M
# rows) and at cosamp_k_max; noiseless Gaussian nonzeros; each request has
# its own Omega and seed.
def serving_requests(n: int, rate: float = 2000.0, seed: int = 0, log_n_lo: int = 14, log_n_hi: int = 20,
                     k_lo: int = 32, k_hi: int = 1024, cosamp_k_max: int = 1024) -> list[dict]:
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    out = []
    for i in range(n):
        N = 1 << int(rng.integers(log_n_lo, log_n_hi + 1))
        M = N // 8
        K = int(min(rng.integers(k_lo, k_hi + 1), M))
        kind = DFT if rng.integers(0, 2) else WHT
        algo = "cosamp" if rng.integers(0, 2) else "omp"
        if algo == "cosamp":
            K = min(K, cosamp_k_max, M // 3)
        out.append({"arrival_s": float(t[i]), "kind": kind, "N": N, "M": M, "K": K, "algo": algo,
                    "seed": seed * 100003 + i + 1})
    return out


def serving_instance(req: dict, prec: str = "fp32") -> tuple[np.ndarray, np.ndarray]:
    """(Omega, y) of one serving request (one instance, noiseless)."""
    inst = make_batch(req["kind"], req["N"], req["M"], req["K"], 1, snr_db=None, prec=prec, seed=req["seed"])
    return inst["omega"], inst["Y"][0]


# The uneven batch: N = 2^e with e uniform over [log_n_lo, log_n_hi]; M = N/4
# or N/8 by a coin; K uniform over [k_lo, k_hi]; partial WHT in FP32 or
# partial DFT in complex64 by a coin; Rademacher or Gaussian nonzeros by a
# coin; noiseless; each instance with its own Omega and seed.
def uneven_batch(n: int, seed: int = 0, log_n_lo: int = 12, log_n_hi: int = 16, k_lo: int = 8,
                 k_hi: int = 256) -> list[dict]:
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        N = 1 << int(rng.integers(log_n_lo, log_n_hi + 1))
        M = N // (4 if rng.integers(0, 2) else 8)
        K = int(min(rng.integers(k_lo, k_hi + 1), M))
        kind = DFT if rng.integers(0, 2) else WHT
        dist = "rademacher" if rng.integers(0, 2) else "gauss"
        out.append({"kind": kind, "N": N, "M": M, "K": K, "dist": dist, "seed": seed * 1000003 + i + 1})
    return out


def uneven_instance(spec: dict) -> tuple[np.ndarray, np.ndarray]:
    """(Omega, y) of one instance of the uneven batch (FP32 working type)."""
    inst = make_batch(spec["kind"], spec["N"], spec["M"], spec["K"], 1, snr_db=None, dist=spec["dist"],
                      prec="fp32", seed=spec["seed"])
    return inst["omega"], inst["Y"][0]
