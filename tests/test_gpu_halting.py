"""Halting on the tolerance (Algorithm 1.1 step 8: ||r_t|| < 1e-6 ||y||) in
FP32 mode, against the FP64 oracle.

The signals have K0 nonzeros and the runs ask for K > K0 columns, noiseless:
the oracle stops on the tolerance after K0 iterations (the residual left is
the FP32 rounding of y, about 3e-8 ||y||), long before K.  FP32 runs must stop
at the same iteration: their downdate of ||r||^2 cannot resolve 1e-6, so the
decision is taken on the explicit residual.  Every kernel that runs OMP is
covered: the persistent one-CTA kernel, the 8-CTA cluster kernel (small
batches), the large-plan sequence, and the uneven-batch launches in shared
and in global memory.  Iteration counts are compared exactly, the reported
||r||/||y|| within the explicit residual's resolution.
"""
import numpy as np
import pytest

import synth
from omp_checks import FP32_RES_BOUND, halting_ambiguous
from oracle import matrices, omp as oomp, transform as tro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1205_4139_gb300 import binding  # noqa: E402


def _ref(kind, N, omega, y, K):
    yv = y.astype(np.complex128 if kind == "dft" else np.float64)
    if N <= 8192:
        return oomp.omp(matrices.sensing_rows(kind, N, omega), yv, K)
    return tro.omp(kind, N, omega, yv, K)


def _check(kind, prec, N, omega, y, K, supp, iters, x, rn):
    ref = _ref(kind, N, omega, y, K)
    near = next((t for t, g in enumerate(ref["gap"]) if g <= 1e-3), len(ref["gap"]))
    got = [int(v) for v in supp[: int(iters)]]
    assert got[:near] == ref["support"][:near]
    if near < len(ref["gap"]) or halting_ambiguous(ref, prec):
        return False
    assert ref["halt"] == "tolerance" and ref["iters"] < K
    assert int(iters) == ref["iters"], (int(iters), ref["iters"])
    rr = ref["resnorm"][-1] / ref["ynorm"]
    assert float(rn) < 1e-6 and abs(float(rn) - rr) <= FP32_RES_BOUND, (float(rn), rr)
    xr = np.asarray(ref["x"])
    assert np.max(np.abs(np.asarray(x)[: len(xr)] - xr)) <= 1e-4 * np.max(np.abs(xr))
    return True


@pytest.mark.parametrize("kind", ["wht", "dft"])
@pytest.mark.parametrize("path", ["fast", "conv", "hybrid"])
@pytest.mark.parametrize("B", [3, 40])  # cluster kernel (B <= 19) and persistent kernel
def test_one_cta_plans_halt_on_tolerance(kind, path, B):
    N, M, K0, K = 1024, 256, 10, 30
    inst = synth.make_batch(kind, N, M, K0, B, prec="fp32", seed=31)
    plan = binding.Plan(N, inst["omega"], kind, "fp32")
    x, supp, iters, rn = (t.cpu().numpy() for t in plan.omp(torch.from_numpy(inst["Y"]).cuda(), K, path=path,
                                                              t_switch=6))
    assert plan.device_error() == 0
    done = sum(_check(kind, "fp32", N, inst["omega"], inst["Y"][b], K, supp[b], iters[b], x[b], rn[b])
               for b in range(min(B, 6)))
    assert done >= 2
    assert (iters < K).all()  # no run went on to K


def test_cluster_equals_persistent_with_halting():
    N, M, K0, K = 2048, 512, 12, 40
    inst = synth.make_batch("dft", N, M, K0, 48, prec="fp32", seed=32)
    plan = binding.Plan(N, inst["omega"], "dft", "fp32")
    y = torch.from_numpy(inst["Y"]).cuda()
    big = plan.omp(y, K, t_switch=8)
    small = plan.omp(y[:4].contiguous(), K, t_switch=8)
    for a, b in zip(big, small):
        assert torch.equal(a[:4], b)


@pytest.mark.parametrize("kind", ["wht", "dft"])
@pytest.mark.parametrize("path", ["fast", "conv", "hybrid"])
def test_large_plans_halt_on_tolerance(kind, path):
    N, M, K0, K = 1 << 14, 2048, 12, 30
    inst = synth.make_batch(kind, N, M, K0, 2, prec="fp32", seed=33)
    plan = binding.Plan(N, inst["omega"], kind, "fp32")
    x, supp, iters, rn = (t.cpu().numpy() for t in plan.omp(torch.from_numpy(inst["Y"]).cuda(), K, path=path,
                                                              t_switch=6))
    assert plan.device_error() == 0
    done = sum(_check(kind, "fp32", N, inst["omega"], inst["Y"][b], K, supp[b], iters[b], x[b], rn[b])
               for b in range(2))
    assert done >= 1


def test_large_plan_fp32_reaches_K_with_accurate_resnorm():
    """A run whose residual reaches the trigger only at t = K: the reported
    ||r||/||y|| comes from the explicit residual."""
    N, M, K = 1 << 15, 4096, 20
    inst = synth.make_batch("dft", N, M, K, 1, prec="fp32", seed=34)
    plan = binding.Plan(N, inst["omega"], "dft", "fp32")
    x, supp, iters, rn = plan.omp(torch.from_numpy(inst["Y"]).cuda(), K)
    ref = _ref("dft", N, inst["omega"], inst["Y"][0], K)
    assert int(iters[0]) == ref["iters"] == K
    assert abs(float(rn[0]) - ref["resnorm"][-1] / ref["ynorm"]) <= FP32_RES_BOUND


@pytest.mark.parametrize("path", ["fast", "conv", "hybrid"])
def test_uneven_batch_halts_on_tolerance(path):
    """cs_omp_batched: shared-memory (N <= 8192), global-memory
    (8192 < N <= 2^16) and large-plan (N > 2^16) instances, each run with
    K > K0."""
    specs = [("wht", 4096, 1024, 9), ("dft", 8192, 1024, 14), ("dft", 1 << 14, 2048, 11),
             ("wht", 1 << 15, 4096, 16), ("dft", 1 << 16, 8192, 20), ("wht", 1 << 17, 8192, 10)]
    plans, ys, Ks, insts = [], [], [], []
    for i, (kind, N, M, K0) in enumerate(specs):
        inst = synth.make_batch(kind, N, M, K0, 1, prec="fp32", seed=40 + i)
        plans.append(binding.Plan(N, inst["omega"], kind, "fp32"))
        ys.append(torch.from_numpy(inst["Y"][0]).cuda())
        Ks.append(K0 + 12)
        insts.append(inst)
    bt = binding.omp_batched(plans, ys, Ks, path=path, t_switch=8)
    torch.cuda.synchronize()
    it, rn = bt.iters.cpu().numpy(), bt.resnorm.cpu().numpy()
    done = 0
    for b, ((kind, N, M, K0), inst) in enumerate(zip(specs, insts)):
        done += _check(kind, "fp32", N, inst["omega"], inst["Y"][0], Ks[b], bt.supp[b].cpu().numpy(), it[b],
                       bt.x[b].cpu().numpy(), rn[b])
    assert done >= 4
    assert plans[0].device_error() == 0
