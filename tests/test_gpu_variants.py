"""The paper's storage variants of c and deterministic row sets through the
same API, on the GPU: half-stored DFT c (conjugate symmetry) and integer WHT c
give the kernel vector of the definition, use less plan memory, and give the
oracle's results (integer c: bit for bit the full-vector plan's); contiguous
and subspace row sets run through the ordinary plan."""
import numpy as np
import pytest

import synth
from oracle import kernelsum, matrices, omp as oomp, transform as tro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1205_4139_gb300 import binding  # noqa: E402

VARIANTS = [("dft", "fp32", "half"), ("dft", "fp64", "half"), ("wht", "fp32", "int"), ("wht", "fp64", "int")]


@pytest.mark.parametrize("kind,prec,store", VARIANTS)
@pytest.mark.parametrize("N,M", [(1024, 300), (8192, 2048), (1 << 15, 5000)])
def test_kernel_vector_and_memory(kind, prec, store, N, M):
    om = synth.draw_omega(N, M, np.random.default_rng(N ^ M))
    full = binding.Plan(N, om, kind, prec)
    var = binding.Plan(N, om, kind, prec, c_storage=store)
    want = tro.kernel_vector(kind, N, om)
    c = var.kernel_vector("fp64").cpu().numpy()
    assert np.max(np.abs(c - want)) < 1e-13
    c32 = var.kernel_vector("fp32").cpu().numpy()
    assert np.max(np.abs(c32 - want)) < 1e-7
    if store == "int":  # exact: identical to the full vector, FP64 and FP32
        assert np.array_equal(c, full.kernel_vector("fp64").cpu().numpy())
        assert np.array_equal(c32, full.kernel_vector("fp32").cpu().numpy())
    else:  # conjugate symmetric by construction
        d = np.arange(N)
        assert np.array_equal(c[(-d) % N], np.conj(c))
    assert var.memory() < full.memory()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("N,M,K", [(1024, 256, 16), (1 << 14, 2048, 24)])
@pytest.mark.parametrize("path", ["fast", "conv", "hybrid"])
def test_int_wht_bit_identical(prec, N, M, K, path):
    inst = synth.make_batch("wht", N, M, K, 8, snr_db=30, prec=prec, seed=N + K)
    y = torch.from_numpy(inst["Y"]).cuda()
    a = binding.Plan(N, inst["omega"], "wht", prec).omp(y, K, path=path, t_switch=8)
    b = binding.Plan(N, inst["omega"], "wht", prec, c_storage="int").omp(y, K, path=path, t_switch=8)
    torch.cuda.synchronize()
    for u, v in zip(a, b):
        assert torch.equal(u, v)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("N,M,K", [(4096, 1024, 32), (1 << 15, 4096, 32)])
def test_half_dft_omp_matches_oracle(prec, N, M, K):
    inst = synth.make_batch("dft", N, M, K, 4, snr_db=None, prec=prec, seed=N + 3)
    plan = binding.Plan(N, inst["omega"], "dft", prec, c_storage="half")
    x, supp, it, rn = plan.omp(torch.from_numpy(inst["Y"]).cuda(), K, path="fast")
    torch.cuda.synchronize()
    supp = supp.cpu().numpy()
    x = x.cpu().numpy()
    for b in range(4):
        ref = tro.omp("dft", N, inst["omega"], inst["Y"][b].astype(np.complex128), K)
        upto = next((t for t, g in enumerate(ref["gap"]) if g <= 1e-3), len(ref["gap"]))
        assert supp[b][:upto].tolist() == ref["support"][:upto]
        if upto == len(ref["gap"]):
            xr = np.asarray(ref["x"])
            assert np.max(np.abs(x[b][: len(xr)] - xr)) < (1e-10 if prec == "fp64" else 1e-4) * np.max(np.abs(xr))
    assert plan.device_error() == 0


@pytest.mark.parametrize("kind,store", [("dft", "half"), ("wht", "int")])
def test_variant_fast_correlation_and_pursuits(kind, store):
    N, M, s = 4096, 1024, 20
    rng = np.random.default_rng(7)
    om = synth.draw_omega(N, M, rng)
    plan = binding.Plan(N, om, kind, "fp64", c_storage=store)
    c = tro.kernel_vector(kind, N, om)
    h0 = (rng.standard_normal((2, N)) + (1j * rng.standard_normal((2, N)) if kind == "dft" else 0)).astype(
        synth.working_dtype(kind, "fp64"))
    supp = np.stack([rng.choice(N, s, replace=False) for _ in range(2)]).astype(np.int32)
    xv = (rng.standard_normal((2, s)) + (1j * rng.standard_normal((2, s)) if kind == "dft" else 0)).astype(h0.dtype)
    h, _ = plan.correlate_fast(torch.from_numpy(h0).cuda(), torch.from_numpy(supp).cuda(), torch.from_numpy(xv).cuda())
    h = h.cpu().numpy()
    for b in range(2):
        want = kernelsum.fast_correlation(kind, N, c, h0[b], supp[b], xv[b])
        assert np.max(np.abs(h[b] - want)) < 1e-12 * np.max(np.abs(want))
    # SP and CoSaMP: same supports as the full-vector plan
    inst = synth.make_batch(kind, N, M, 8, 6, snr_db=None, prec="fp64", seed=5)
    y = torch.from_numpy(inst["Y"]).cuda()
    full = binding.Plan(N, inst["omega"], kind, "fp64")
    var = binding.Plan(N, inst["omega"], kind, "fp64", c_storage=store)
    for algo in ("sp", "cosamp"):
        a = full.pursuit(algo, y, 8)
        b = var.pursuit(algo, y, 8)
        torch.cuda.synchronize()
        assert torch.equal(a[1], b[1])
        assert np.max(np.abs(a[0].cpu().numpy() - b[0].cpu().numpy())) < 1e-10


def test_deterministic_row_sets():
    """Omega built deterministically goes through the same API: a contiguous
    (low-pass) DFT row set and a WHT row set that is a linear subspace."""
    N, M, K = 1024, 256, 8
    om = np.arange(M, dtype=np.int32)
    plan = binding.Plan(N, om, "dft", "fp64")
    c = plan.kernel_vector("fp64").cpu().numpy()
    assert np.max(np.abs(c - tro.kernel_vector("dft", N, om))) < 1e-13
    rng = np.random.default_rng(3)
    sup = np.sort(rng.choice(N, K, replace=False))
    xv = rng.standard_normal(K) + 1j * rng.standard_normal(K)
    y = synth.measure("dft", N, om, sup.astype(np.int32), xv)
    x, s, it, rn = plan.omp(torch.from_numpy(y[None]).cuda(), K)
    Phi = matrices.sensing("dft", N, om)
    ref = oomp.omp(Phi, y, K)
    upto = next((t for t, g in enumerate(ref["gap"]) if g <= 1e-3), len(ref["gap"]))
    assert s.cpu().numpy()[0][:upto].tolist() == ref["support"][:upto]

    basis = [0b0000000011, 0b0000111100, 0b1101000000, 0b0010010001, 0b0100001000, 0b0001100110]
    span = {0}
    for v in basis:
        span |= {q ^ v for q in span}
    om2 = np.array(sorted(span), dtype=np.int32)
    for store in ("full", "int"):
        p2 = binding.Plan(N, om2, "wht", "fp64", c_storage=store)
        c2 = p2.kernel_vector("fp64").cpu().numpy()
        assert np.array_equal(c2, tro.kernel_vector("wht", N, om2))
