"""Per-iteration flop counts of Table I (Sec. III-B) and the quantities the
paper derives from them (Sec. IV).

The paper counts one complex multiplication as 6 flops and one complex
addition as 2 flops (Sec. III-B).  Iteration t computes h_{t-1}:

    partial Fourier   conventional 5 N log2 N      fast: t=1 5 N log2 N, t>1 6 N (t-1)
    partial Hadamard  conventional 2 N log2 N      fast: t=1 2 N log2 N, t>1 2 N (t-1)

The "excessive point" (Sec. IV) is the last iteration at which the fast form
costs no more than the transform; the paper switches to the conventional
correlation from the next iteration on.  For fast CoSaMP every iteration but
the first correlates against the K atoms of the current estimate, so its
per-iteration cost against one transform is 6 N K / (5 N log2 N) (Sec. IV).
"""
from __future__ import annotations

import math


def conventional_flops(kind: str, N: int) -> float:
    n = math.log2(N)
    return (5.0 if kind == "dft" else 2.0) * N * n


def fast_flops(kind: str, N: int, t: int) -> float:
    if t <= 1:
        return conventional_flops(kind, N)
    return (6.0 if kind == "dft" else 2.0) * N * (t - 1)


def excessive_point(kind: str, N: int) -> int:
    """Largest t with fast_flops(t) <= conventional_flops (Sec. IV)."""
    t = 1
    while fast_flops(kind, N, t + 1) <= conventional_flops(kind, N):
        t += 1
    return t


def omp_correlation_flops(kind: str, N: int, iters: int, t_switch: int) -> float:
    """Paper-model correlation flops of one OMP run of ``iters`` iterations
    that uses the fast form while t <= t_switch and the transform after."""
    total = 0.0
    for t in range(1, iters + 1):
        total += fast_flops(kind, N, t) if t <= t_switch else conventional_flops(kind, N)
    return total


def cosamp_fast_ratio(N: int, K: int) -> float:
    """Per-iteration cost of fast over conventional CoSaMP, partial Fourier."""
    return 6.0 * N * K / conventional_flops("dft", N)
