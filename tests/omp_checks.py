"""Shared comparison rules of the GPU OMP tests against the FP64 oracle.

Halting (Algorithm 1.1 step 8: t = K or ||r_t|| < rel_tol ||y||).  FP64 runs
decide on the FP64 downdate of ||r||^2, which resolves ||r||/||y|| to about
1e-8.  FP32 runs decide on the explicit residual y - Phi x whenever the
downdate comes near the tolerance; formed in FP32 with FP64 accumulation it
resolves ||r||/||y|| to a few 1e-7 (FP32_RES_BOUND).  A halting decision is
compared exactly unless the oracle's ||r_t||/||y|| at some iteration lies
within that resolution of the tolerance (FP64: within 1e-3 relative of it).
"""
FP32_RES_BOUND = 5e-7


def halting_ambiguous(ref, prec, rel_tol=1e-6):
    bound = 1e-3 * rel_tol if prec == "fp64" else FP32_RES_BOUND
    yn = ref["ynorm"]
    return yn > 0 and any(abs(rn / yn - rel_tol) <= bound for rn in ref["resnorm"])


def resnorm_tol(rr, prec):
    """Allowed |reported - oracle| for ||r||/||y|| = rr at exit.  FP64: the
    downdate.  FP32: the explicit residual where the downdate came near the
    tolerance (rr small), else the downdate, whose ||r||^2 carries about 1e-6
    of FP32 rounding of h_0 on the right-hand side."""
    if prec == "fp64":
        return 1e-6 * rr + 1e-7
    return FP32_RES_BOUND + (2e-6 / rr if rr > 2e-3 else 0.0)
