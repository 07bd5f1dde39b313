"""Subspace pursuit and CoSaMP on the GPU (through the C ABI) against the
FP64 oracle.  Supports must match exactly wherever the oracle's selections
are not near ties; coefficients within 1e-10 (FP64) or 1e-4 (FP32)
relative in noiseless cases."""
import numpy as np
import pytest

import synth
from oracle import matrices, pursuits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1205_4139_gb300 import binding  # noqa: E402

MODES = [("wht", "fp64"), ("wht", "fp32"), ("dft", "fp64"), ("dft", "fp32")]


def run_and_check(inst, algo, path, prec, noiseless=True):
    kind, N, K = inst["kind"], inst["N"], inst["K"]
    plan = binding.Plan(N, inst["omega"], kind, prec)
    x, supp, iters, rn = (t.cpu().numpy() for t in plan.pursuit(algo, torch.from_numpy(inst["Y"]).cuda(), K,
                                                                  path=path))
    Phi = matrices.sensing_rows(kind, N, inst["omega"])
    for b in range(inst["B"]):
        yb = inst["Y"][b].astype(np.complex128 if kind == "dft" else np.float64)
        ref = pursuits.subspace_pursuit(Phi, yb, K) if algo == "sp" else pursuits.cosamp(Phi, yb, K)
        got = [j for j in supp[b].tolist() if j >= 0]
        assert got == ref["support"].tolist(), (algo, b, got, ref["support"].tolist())
        xr = np.asarray(ref["x"])
        if noiseless and len(xr):
            err = np.max(np.abs(x[b][: len(xr)] - xr)) / np.max(np.abs(xr))
            assert err < (1e-10 if prec == "fp64" else 1e-4), (algo, b, err)
    return iters


@pytest.mark.parametrize("kind,prec", MODES)
@pytest.mark.parametrize("algo", ["sp", "cosamp"])
@pytest.mark.parametrize("path", ["fast", "conv"])
def test_pursuit_noiseless_recovery(kind, prec, algo, path):
    inst = synth.make_batch(kind, 512, 192, 10, 4, snr_db=None, prec=prec, seed=41)
    iters = run_and_check(inst, algo, path, prec)
    assert (iters >= 1).all()


@pytest.mark.parametrize("algo", ["sp", "cosamp"])
def test_pursuit_dft_c64_noisy(algo):
    """Partial DFT complex64, N=4096, M=1024, 40 dB (the benchmark's row set);
    K = 32 keeps the oracle quick."""
    inst = synth.make_batch("dft", 4096, 1024, 32, 3, snr_db=40.0, prec="fp32", seed=5)
    run_and_check(inst, algo, "fast", "fp32", noiseless=False)


def test_cosamp_small_fourier_case():
    """The case the paper quotes for fast CoSaMP: M = 64, N = 8192, K = 4."""
    inst = synth.make_batch("dft", 8192, 64, 4, 3, snr_db=None, prec="fp64", seed=2)
    run_and_check(inst, "cosamp", "fast", "fp64")


def test_pursuit_rejects_sizes():
    plan = binding.Plan(64, np.arange(0, 64, 2, dtype=np.int32), "dft", "fp32")
    y = torch.zeros(1, 32, dtype=torch.complex64, device="cuda")
    with pytest.raises(binding.CsError):
        plan.pursuit("cosamp", y, 11)   # 3K > M
    with pytest.raises(binding.CsError):
        plan.pursuit("sp", y, 17)       # 2K > M
    x, supp, iters, rn = plan.pursuit("sp", y, 4)   # zero measurement: no iteration
    assert int(iters[0]) == 0 and (supp.cpu().numpy() == -1).all()


@pytest.mark.parametrize("kind,prec", MODES)
@pytest.mark.parametrize("algo", ["sp", "cosamp"])
@pytest.mark.parametrize("path", ["fast", "conv"])
def test_pursuit_cg_noiseless(kind, prec, algo, path):
    """K = 64 on one-CTA plans: column sets of 128 (SP) and 192 (CoSaMP)
    take the conjugate-gradient least squares; supports, iteration counts
    and coefficients as the oracle's (dense Cholesky solves)."""
    inst = synth.make_batch(kind, 4096, 1024, 64, 2, snr_db=None, prec=prec, seed=43)
    run_and_check(inst, algo, path, prec)


@pytest.mark.parametrize("algo", ["sp", "cosamp"])
def test_pursuit_cg_dft_c64_noisy(algo):
    """The benchmark's SP workload shape (partial DFT complex64, N = 4096,
    M = 1024, K = 64, 40 dB) against the oracle, least squares by conjugate
    gradients."""
    inst = synth.make_batch("dft", 4096, 1024, 64, 3, snr_db=40.0, prec="fp32", seed=7)
    run_and_check(inst, algo, "fast", "fp32", noiseless=False)
