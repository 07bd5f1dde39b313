"""Subspace pursuit and CoSaMP on large plans (N > 8192: correlation over the
GPU, two-stage top-k over N, one CTA per instance for the least squares)
against the transform-based FP64 oracle of the same standard forms."""
import numpy as np
import pytest

import synth
from oracle import transform as tro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1205_4139_gb300 import binding  # noqa: E402

MODES = [("wht", "fp64"), ("wht", "fp32"), ("dft", "fp64"), ("dft", "fp32")]


@pytest.mark.parametrize("kind,prec", MODES)
@pytest.mark.parametrize("algo", ["sp", "cosamp"])
@pytest.mark.parametrize("path", ["fast", "conv"])
def test_large_pursuit_noiseless_matches_oracle(kind, prec, algo, path):
    N, M, K = 1 << 14, 2048, 16
    inst = synth.make_batch(kind, N, M, K, 3, snr_db=None, prec=prec, seed=40 + K)
    plan = binding.Plan(N, inst["omega"], kind, prec)
    x, supp, it, rn = plan.pursuit(algo, torch.from_numpy(inst["Y"]).cuda(), K, path=path)
    torch.cuda.synchronize()
    x, supp, it = x.cpu().numpy(), supp.cpu().numpy(), it.cpu().numpy()
    wt = np.complex128 if kind == "dft" else np.float64
    f = tro.subspace_pursuit if algo == "sp" else tro.cosamp
    for b in range(3):
        ref = f(kind, N, inst["omega"], inst["Y"][b].astype(wt), K)
        assert supp[b].tolist() == list(ref["support"])
        assert sorted(ref["support"].tolist()) == sorted(inst["support"][b].tolist())
        xr = np.asarray(ref["x"])
        assert np.max(np.abs(x[b] - xr)) < (1e-10 if prec == "fp64" else 1e-4) * np.max(np.abs(xr))
        if prec == "fp64":
            assert it[b] == ref["iters"]
    assert plan.device_error() == 0


@pytest.mark.parametrize("kind", ["dft", "wht"])
@pytest.mark.parametrize("algo", ["sp", "cosamp"])
def test_large_pursuit_noisy_fp64(kind, algo):
    """40 dB, FP64: same iterations and supports as the oracle (no near ties
    in these seeded cases), residual norms within rounding."""
    N, M, K = 1 << 15, 4096, 24
    inst = synth.make_batch(kind, N, M, K, 2, snr_db=40, prec="fp64", seed=5)
    plan = binding.Plan(N, inst["omega"], kind, "fp64")
    x, supp, it, rn = plan.pursuit(algo, torch.from_numpy(inst["Y"]).cuda(), K, path="fast")
    torch.cuda.synchronize()
    f = tro.subspace_pursuit if algo == "sp" else tro.cosamp
    for b in range(2):
        ref = f(kind, N, inst["omega"], inst["Y"][b], K)
        assert supp.cpu().numpy()[b].tolist() == list(ref["support"])
        assert int(it[b]) == ref["iters"]
        assert abs(float(rn[b]) - ref["resnorm"][-1] / ref["ynorm"]) < 1e-8


def test_large_pursuit_zero_measurement_and_batch():
    N, M, K = 1 << 14, 2048, 8
    inst = synth.make_batch("dft", N, M, K, 4, snr_db=None, prec="fp32", seed=8)
    Y = inst["Y"].copy()
    Y[2] = 0
    plan = binding.Plan(N, inst["omega"], "dft", "fp32")
    for algo in ("sp", "cosamp"):
        x, s, it, rn = plan.pursuit(algo, torch.from_numpy(Y).cuda(), K)
        s = s.cpu().numpy()
        assert (s[2] == -1).all() and int(it[2]) == 0 and float(rn[2]) == 0.0
        for b in (0, 1, 3):
            assert sorted(s[b].tolist()) == sorted(inst["support"][b].tolist())
