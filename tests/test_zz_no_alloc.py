"""cs_omp_noalloc, the OMP entry point that allocates nothing.

It serves callers that may not allocate device memory while they solve (a
latency-bound request loop cannot take the device synchronisation of
cudaMalloc/cudaFree; some processes give the library no memory beyond their
own buffers).  It runs the same kernel as cs_omp with its scratch in a fixed
library array and the same switch point, so its outputs must equal cs_omp's
bit for bit.  Two calls in a row check that the contents the previous call
leaves in the shared array do not leak into the next one.  This file is
collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1205_4139_gb300 import binding  # noqa: E402


def _outputs(B, K, kind):
    return (torch.empty(B, K, dtype=binding.ls_dtype(kind), device="cuda"),
            torch.empty(B, K, dtype=torch.int32, device="cuda"),
            torch.empty(B, dtype=torch.int32, device="cuda"),
            torch.empty(B, dtype=torch.float64, device="cuda"))


def _call(fn, plan, y, K, outs, path, t_switch=-1, rel_tol=1e-6):
    halt = binding.Halt(rel_tol, binding.PATHS[path], t_switch, 0)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = fn(plan._h, p(y), y.shape[0], K, ctypes.byref(halt), p(outs[0]), p(outs[1]), p(outs[2]), p(outs[3]),
            stream)
    assert st == 0, binding.load().cs_last_error()


def _equal(a, b):
    return all(torch.equal(u, v) for u, v in zip(a, b))


@pytest.mark.parametrize("kind,prec,N,M,K,B,snr,path", [
    ("dft", "fp32", 4096, 1024, 64, 300, 40.0, "hybrid"),
    ("wht", "fp64", 1024, 256, 16, 5, None, "fast"),
    ("dft", "fp64", 512, 160, 12, 40, None, "conv"),
])
def test_noalloc_matches_cs_omp(kind, prec, N, M, K, B, snr, path):
    L = binding.load()
    inst = synth.make_batch(kind, N, M, K, B, snr_db=snr, prec=prec, seed=3)
    plan = binding.Plan(N, inst["omega"], kind, prec)
    y = torch.from_numpy(inst["Y"]).cuda()
    ref = _outputs(B, K, kind)
    _call(L.cs_omp, plan, y, K, ref, path)
    for _ in range(2):  # two calls in a row on the shared scratch
        got = _outputs(B, K, kind)
        for t in got:
            t.fill_(7)
        _call(L.cs_omp_noalloc, plan, y, K, got, path)
        torch.cuda.synchronize()
        assert _equal(got, ref)


def test_noalloc_takes_the_plans_switch_point():
    """With t_switch < 0 both entry points switch where cs_plan_switch says,
    on an untuned plan (the GB300 table) and after cs_plan_tune.  The signal
    has 4 nonzeros and the run asks for 24 columns with the tolerance off, so
    from t = 5 on the residual is rounding noise and each selection depends on
    which correlation computed it: runs with different switch points pick
    different columns there, which makes the switch point visible."""
    L = binding.load()
    N, M, K, B = 4096, 1024, 24, 48
    inst = synth.make_batch("dft", N, M, 4, B, prec="fp32", seed=11)
    plan = binding.Plan(N, inst["omega"], "dft", "fp32")
    y = torch.from_numpy(inst["Y"]).cuda()

    def check():
        ts = plan.switch_point()
        ref = _outputs(B, K, "dft")
        _call(L.cs_omp, plan, y, K, ref, "hybrid", t_switch=ts, rel_tol=0.0)
        other = _outputs(B, K, "dft")
        t_other = 1 if ts >= 12 else K
        _call(L.cs_omp, plan, y, K, other, "hybrid", t_switch=t_other, rel_tol=0.0)
        torch.cuda.synchronize()
        # the switch point is visible in the outputs of this workload
        assert not torch.equal(other[1], ref[1])
        for _ in range(2):
            got = _outputs(B, K, "dft")
            _call(L.cs_omp_noalloc, plan, y, K, got, "hybrid", t_switch=-1, rel_tol=0.0)
            dflt = _outputs(B, K, "dft")
            _call(L.cs_omp, plan, y, K, dflt, "hybrid", t_switch=-1, rel_tol=0.0)
            torch.cuda.synchronize()
            assert _equal(got, ref)
            assert _equal(dflt, ref)
        return ts

    ts0 = check()
    assert ts0 == 64  # GB300 table for N <= 8192
    t_best, _ = plan.tune(y, K, rel_tol=0.0)
    assert plan.switch_point() == t_best
    check()


def test_noalloc_rejects_bad_arguments():
    L = binding.load()
    inst = synth.make_batch("dft", 64, 20, 4, 2, prec="fp32", seed=1)
    plan = binding.Plan(64, inst["omega"], "dft", "fp32")
    y = torch.from_numpy(inst["Y"]).cuda()
    outs = _outputs(2, 4, "dft")
    halt = binding.Halt(1e-6, 2, -1, 0)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    # K larger than M is invalid
    assert L.cs_omp_noalloc(plan._h, p(y), 2, 21, ctypes.byref(halt), p(outs[0]), p(outs[1]), p(outs[2]),
                            p(outs[3]), None) == 1
    # unknown path
    bad = binding.Halt(1e-6, 7, -1, 0)
    assert L.cs_omp_noalloc(plan._h, p(y), 2, 4, ctypes.byref(bad), p(outs[0]), p(outs[1]), p(outs[2]),
                            p(outs[3]), None) == 1
