"""Subspace pursuit and CoSaMP on large plans with least-squares sets of more
than 96 columns, which the library solves by FP64 conjugate gradients on a
thread-block cluster (Gram products read off the kernel vector) instead of
appending the columns to a Cholesky factor.  Compared with the transform
oracle of the same standard forms (a dense Cholesky solve of the explicitly
formed Gram matrix) where the oracle finishes in seconds, and by exact
recovery of the generating support at K up to 1024."""
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


def _oracle(algo):
    return tro.subspace_pursuit if algo == "sp" else tro.cosamp


@pytest.mark.parametrize("kind,prec", MODES)
@pytest.mark.parametrize("algo", ["sp", "cosamp"])
@pytest.mark.parametrize("path", ["fast", "conv"])
def test_cg_pursuit_noiseless_matches_oracle(kind, prec, algo, path):
    """K = 64 (SP sets of 128 columns, CoSaMP 192): supports, iteration counts
    (FP64) and coefficients against the oracle."""
    N, M, K = 1 << 14, 2048, 64
    inst = synth.make_batch(kind, N, M, K, 2, snr_db=None, prec=prec, seed=70)
    plan = binding.Plan(N, inst["omega"], kind, prec)
    x, supp, it, rn = plan.pursuit(algo, torch.from_numpy(inst["Y"]).cuda(), K, path=path)
    torch.cuda.synchronize()
    x, supp, it = x.cpu().numpy(), supp.cpu().numpy(), it.cpu().numpy()
    wt = np.complex128 if kind == "dft" else np.float64
    for b in range(2):
        ref = _oracle(algo)(kind, N, inst["omega"], inst["Y"][b].astype(wt), K)
        assert supp[b].tolist() == list(ref["support"]), b
        assert sorted(ref["support"].tolist()) == sorted(inst["support"][b].tolist())
        xr = np.asarray(ref["x"])
        err = np.max(np.abs(x[b] - xr)) / np.max(np.abs(xr))
        assert err < (1e-10 if prec == "fp64" else 1e-4), (b, err)
        if prec == "fp64":
            assert it[b] == ref["iters"]
    assert plan.device_error() == 0


@pytest.mark.parametrize("kind", ["dft", "wht"])
@pytest.mark.parametrize("algo", ["sp", "cosamp"])
def test_cg_pursuit_noisy_fp64_matches_oracle(kind, algo):
    """40 dB, FP64, K = 40 (CoSaMP sets of 120 columns, SP 80 by the Cholesky
    append) and K = 72 (both by conjugate gradients): iterations, supports and
    residual norms as the oracle's."""
    N, M = 1 << 14, 2048
    for K in (40, 72):
        inst = synth.make_batch(kind, N, M, K, 2, snr_db=40, prec="fp64", seed=6 + K)
        plan = binding.Plan(N, inst["omega"], kind, "fp64")
        x, supp, it, rn = plan.pursuit(algo, torch.from_numpy(inst["Y"]).cuda(), K, path="fast")
        torch.cuda.synchronize()
        for b in range(2):
            ref = _oracle(algo)(kind, N, inst["omega"], inst["Y"][b], K)
            assert supp.cpu().numpy()[b].tolist() == list(ref["support"]), (K, b)
            assert int(it[b]) == ref["iters"], (K, b)
            assert abs(float(rn[b]) - ref["resnorm"][-1] / ref["ynorm"]) < 1e-8, (K, b)
        assert plan.device_error() == 0


@pytest.mark.parametrize("algo,N,M,K", [("cosamp", 1 << 15, 8192, 256), ("sp", 1 << 15, 8192, 384),
                                        ("cosamp", 1 << 17, 1 << 15, 1024), ("sp", 1 << 17, 1 << 15, 1024)])
def test_cg_pursuit_large_k_recovers(algo, N, M, K):
    """Noiseless DFT complex64 at K up to 1024 (sets of up to 3072 columns):
    the generating support is recovered exactly, x to 1e-4 relative, and the
    reported residual norm agrees with ||y - Phi_S x|| recomputed in FP64."""
    inst = synth.make_batch("dft", N, M, K, 1, snr_db=None, prec="fp32", seed=91)
    plan = binding.Plan(N, inst["omega"], "dft", "fp32")
    x, supp, it, rn = plan.pursuit(algo, torch.from_numpy(inst["Y"]).cuda(), K)
    torch.cuda.synchronize()
    s = supp.cpu().numpy()[0]
    assert sorted(s.tolist()) == sorted(inst["support"][0].tolist())
    order = np.argsort(inst["support"][0])
    xt = inst["values"][0][order]
    xg = x.cpu().numpy()[0]
    assert np.max(np.abs(xg - xt)) < 1e-4 * np.max(np.abs(xt))
    y = inst["Y"][0].astype(np.complex128)
    r = y - tro.synthesize("dft", N, inst["omega"], s, xg)
    assert abs(float(rn[0]) - np.linalg.norm(r) / np.linalg.norm(y)) < 1e-6
    assert 1 <= int(it[0]) <= (K if algo == "sp" else 50)
    assert plan.device_error() == 0


def test_cg_pursuit_limits():
    """K <= 1024 on large plans, K <= 128 on one-CTA plans (unsupported
    beyond), and the set-size rules of each algorithm (invalid beyond)."""
    N, M = 1 << 14, 4096
    inst = synth.make_batch("wht", N, M, 8, 1, snr_db=None, prec="fp32", seed=3)
    plan = binding.Plan(N, inst["omega"], "wht", "fp32")
    y = torch.from_numpy(inst["Y"]).cuda()
    with pytest.raises(binding.CsError, match="invalid argument"):
        plan.pursuit("cosamp", y, 1366)  # 3K > M
    inst2 = synth.make_batch("wht", 1 << 17, 1 << 15, 8, 1, snr_db=None, prec="fp32", seed=3)
    plan2 = binding.Plan(1 << 17, inst2["omega"], "wht", "fp32")
    with pytest.raises(binding.CsError, match="beyond the kernels"):
        plan2.pursuit("sp", torch.from_numpy(inst2["Y"]).cuda(), 1025)
    small = synth.make_batch("wht", 4096, 2048, 8, 1, snr_db=None, prec="fp32", seed=3)
    plan3 = binding.Plan(4096, small["omega"], "wht", "fp32")
    with pytest.raises(binding.CsError, match="beyond the kernels"):
        plan3.pursuit("sp", torch.from_numpy(small["Y"]).cuda(), 129)


@pytest.mark.parametrize("N,M", [(4096, 512), (1 << 14, 2048)])
def test_cg_dependent_columns_end(N, M):
    """A WHT row set that is a linear subspace (Omega = {0 .. M-1}): columns
    j and j' coincide whenever j ^ j' has no low bits, so CoSaMP's candidate
    sets hold whole groups of equal columns and their Gram matrices are
    singular.  The conjugate-gradient least squares must still end (its
    iteration bound), with finite outputs and a clean status word, on both
    plan sizes."""
    rng = np.random.default_rng(4)
    omega = np.arange(M, dtype=np.int32)
    K = 40
    sup = np.sort(rng.choice(N, K, replace=False))
    y = synth.measure("wht", N, omega, sup, rng.standard_normal(K))[None].astype(np.float64)
    plan = binding.Plan(N, omega, "wht", "fp64")
    x, supp, it, rn = plan.pursuit("cosamp", torch.from_numpy(y).cuda(), K, max_iter=6)
    torch.cuda.synchronize()
    assert np.isfinite(x.cpu().numpy()).all() and np.isfinite(float(rn[0]))
    assert 1 <= int(it[0]) <= 6
    assert plan.device_error() == 0


def test_pursuit_into_a_captured_graph():
    """SP on a large plan with K = 96 (97 iterations allowed: eligible for
    the device-side loop) called while the stream is being captured: the
    iterations go into the caller's graph instead, and replaying it gives
    the eager call's results bit for bit."""
    N, M, K = 1 << 14, 2048, 96
    inst = synth.make_batch("dft", N, M, K, 2, snr_db=None, prec="fp32", seed=31)
    plan = binding.Plan(N, inst["omega"], "dft", "fp32")
    y = torch.from_numpy(inst["Y"]).cuda()
    x0, s0, i0, r0 = plan.pursuit("sp", y, K)  # eager: also grows the plan's workspace
    torch.cuda.synchronize()
    x = torch.zeros_like(x0)
    s = torch.zeros_like(s0)
    it = torch.zeros_like(i0)
    rn = torch.zeros_like(r0)
    st = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st, capture_error_mode="relaxed"):
        plan.pursuit_into("sp", y, K, x, s, it, rn, stream=st)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(s, s0) and torch.equal(x, x0) and torch.equal(it, i0) and torch.equal(rn, r0)
    assert plan.device_error() == 0
