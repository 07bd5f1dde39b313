"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: FP64 mode h within 1e-12 relative (l_inf / ||h||_inf), FP32 mode
within 2e-5; supports bit-exact up to the first iteration whose oracle
top-two |h| gap is at most 1e-3 relative; recovered x within 1e-10 (FP64) or
1e-4 (FP32) relative in noiseless cases.
"""
import numpy as np
import pytest

import synth
from omp_checks import halting_ambiguous, resnorm_tol
from oracle import kernelsum, matrices, omp as oomp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1205_4139_gb300 import binding  # noqa: E402

TOL_H = {"fp64": 1e-12, "fp32": 2e-5}
MODES = [("wht", "fp64"), ("wht", "fp32"), ("dft", "fp64"), ("dft", "fp32")]


def np_dtype(kind, prec):
    return synth.working_dtype(kind, prec)


def rel_inf(a, b):
    den = np.max(np.abs(b))
    return np.max(np.abs(a - b)) / (den if den > 0 else 1.0)


def rand_work(rng, shape, kind, prec):
    v = rng.standard_normal(shape) + (1j * rng.standard_normal(shape) if kind == "dft" else 0)
    return v.astype(np_dtype(kind, prec))


def omega_for(N, M, seed):
    return synth.draw_omega(N, M, np.random.default_rng(seed))


def phi_rows(kind, N, om):
    return matrices.sensing_rows(kind, N, om)


# ------------------------------------------------------------- kernel vector
@pytest.mark.parametrize("kind,prec", MODES)
@pytest.mark.parametrize("N,M", [(1, 1), (2, 1), (16, 5), (64, 64), (1024, 256), (4096, 1024), (8192, 777)])
def test_kernel_vector(kind, prec, N, M):
    om = omega_for(N, M, N + M)
    plan = binding.Plan(N, om, kind, prec)
    c = plan.kernel_vector("fp64").cpu().numpy()
    want = kernelsum.kernel_vector_rows(kind, N, om)
    assert np.max(np.abs(c - want)) < 1e-13
    if kind == "wht":  # N c is an exact integer on the GPU too
        assert np.array_equal(N * c, np.round(N * want))
    c32 = plan.kernel_vector("fp32").cpu().numpy()
    assert np.max(np.abs(c32 - want)) < 1e-7 * max(1.0, np.max(np.abs(want)))
    assert plan.info()["N"] == N


def test_empty_omega():
    plan = binding.Plan(64, np.zeros(0, np.int32), "dft", "fp32")
    c = plan.kernel_vector("fp64").cpu().numpy()
    assert np.all(c == 0)


# --------------------------------------------------- conventional correlation
@pytest.mark.parametrize("kind,prec", MODES)
@pytest.mark.parametrize("N,M,B", [(2, 2, 3), (16, 7, 5), (256, 100, 4), (1024, 333, 3), (4096, 1024, 2),
                                   (8192, 2000, 2)])
def test_correlate(kind, prec, N, M, B):
    rng = np.random.default_rng(N * 7 + M)
    om = omega_for(N, M, N + 3 * M)
    plan = binding.Plan(N, om, kind, prec)
    r = rand_work(rng, (B, M), kind, prec)
    h, am = plan.correlate(torch.from_numpy(r).cuda())
    h = h.cpu().numpy()
    am = am.cpu().numpy()
    Phi = phi_rows(kind, N, om)
    for b in range(B):
        want = oomp.correlate(Phi, r[b].astype(np.complex128))
        if kind == "wht":
            want = want.real
        assert rel_inf(h[b], want) < TOL_H[prec], (b, rel_inf(h[b], want))
        j, gap = oomp.identify(want, [])
        if gap > 1e-3:
            assert am[b] == j


# ------------------------------------------------------------ fast correlation
@pytest.mark.parametrize("kind,prec", MODES)
@pytest.mark.parametrize("N,M,s,B", [(2, 1, 1, 2), (16, 9, 3, 4), (512, 200, 0, 2), (1024, 256, 15, 3),
                                     (4096, 1024, 63, 3), (8192, 1500, 40, 2)])
def test_correlate_fast(kind, prec, N, M, s, B):
    rng = np.random.default_rng(N + s)
    om = omega_for(N, M, N * 5 + M)
    plan = binding.Plan(N, om, kind, prec)
    c = kernelsum.kernel_vector_rows(kind, N, om)
    h0 = rand_work(rng, (B, N), kind, prec)
    supp = np.stack([synth.draw_support(N, s, rng) for _ in range(B)]).astype(np.int32).reshape(B, s)
    x = rand_work(rng, (B, s), kind, prec)
    h, am = plan.correlate_fast(torch.from_numpy(h0).cuda(), torch.from_numpy(supp).cuda(), torch.from_numpy(x).cuda())
    h = h.cpu().numpy()
    am = am.cpu().numpy()
    for b in range(B):
        wt = np.complex128 if kind == "dft" else np.float64
        want = kernelsum.fast_correlation(kind, N, c, h0[b].astype(wt), supp[b], x[b].astype(wt))
        if kind == "wht":
            want = want.real
        assert rel_inf(h[b], want) < TOL_H[prec], (b, rel_inf(h[b], want))
        j, gap = oomp.identify(want, supp[b].tolist())
        if gap > 1e-3:
            assert am[b] == j


def test_fast_equals_conventional_on_gpu():
    """Sec. III-A exactness on the GPU: the two correlations agree."""
    kind, prec, N, M, s = "dft", "fp64", 1024, 300, 12
    rng = np.random.default_rng(3)
    om = omega_for(N, M, 9)
    plan = binding.Plan(N, om, kind, prec)
    y = rand_work(rng, (1, M), kind, prec)
    supp = synth.draw_support(N, s, rng).astype(np.int32)[None]
    x = rand_work(rng, (1, s), kind, prec)
    Phi = phi_rows(kind, N, om)
    r = y[0] - Phi[:, supp[0]] @ x[0]
    h_conv, _ = plan.correlate(torch.from_numpy(r[None]).cuda())
    h0, _ = plan.correlate(torch.from_numpy(y).cuda())
    h_fast, _ = plan.correlate_fast(h0, torch.from_numpy(supp).cuda(), torch.from_numpy(x).cuda())
    assert rel_inf(h_fast.cpu().numpy(), h_conv.cpu().numpy()) < 1e-12


# ------------------------------------------------------------------------ OMP
def check_omp(inst, res, prec, noiseless, x_tol=None, check_all=True):
    kind, N = inst["kind"], inst["N"]
    Phi = phi_rows(kind, N, inst["omega"])
    x, supp, iters, rn = (t.cpu().numpy() for t in res)
    K = inst["K"]
    B = inst["B"] if check_all else min(inst["B"], 3)
    for b in range(B):
        yb = inst["Y"][b].astype(np.complex128 if kind == "dft" else np.float64)
        ref = oomp.omp(Phi, yb, K)
        # first iteration whose identification is a near tie
        near = next((t for t, g in enumerate(ref["gap"]) if g <= 1e-3), len(ref["gap"]))
        got = supp[b][: iters[b]].tolist()
        assert got[:near] == ref["support"][:near], (b, near, got, ref["support"])
        if near == len(ref["gap"]):
            assert iters[b] == ref["iters"] or halting_ambiguous(ref, prec), (b, iters[b], ref["iters"])
            xr = np.asarray(ref["x"])
            err = np.max(np.abs(x[b][: len(xr)] - xr)) / np.max(np.abs(xr))
            tol = x_tol if x_tol is not None else (1e-10 if prec == "fp64" else 1e-4)
            assert err < tol, (b, err)
            assert np.all(supp[b][iters[b]:] == -1)
            rr = ref["resnorm"][-1] / ref["ynorm"]
            assert abs(rn[b] - rr) <= resnorm_tol(rr, prec), (b, rn[b], rr)


@pytest.mark.parametrize("path", ["fast", "conv", "hybrid"])
def test_omp_wht_fp64_single(path):
    """Partial WHT, FP64, N=1024, M=256, K=16, noiseless, seed 0."""
    inst = synth.make_batch(**synth.CONFIG_WHT_FP64_SINGLE)
    plan = binding.Plan(inst["N"], inst["omega"], "wht", "fp64")
    res = plan.omp(torch.from_numpy(inst["Y"]).cuda(), inst["K"], path=path)
    assert plan.device_error() == 0
    check_omp(inst, res, "fp64", True)
    # exact recovery of the drawn signal
    x, supp, iters, _ = (t.cpu().numpy() for t in res)
    assert sorted(supp[0][: iters[0]].tolist()) == sorted(inst["support"][0].tolist())


@pytest.mark.parametrize("kind,prec", MODES)
@pytest.mark.parametrize("path", ["fast", "conv", "hybrid"])
def test_omp_small_batches(kind, prec, path):
    inst = synth.make_batch(kind, 512, 160, 12, 5, snr_db=None, prec=prec, seed=21)
    plan = binding.Plan(512, inst["omega"], kind, prec)
    res = plan.omp(torch.from_numpy(inst["Y"]).cuda(), 12, path=path)
    assert plan.device_error() == 0
    check_omp(inst, res, prec, True)


@pytest.mark.parametrize("path", ["fast", "conv", "hybrid"])
def test_omp_dft_c64_noisy_batch(path):
    """Partial DFT complex64, N=4096, M=1024, K=64, 40 dB (a slice of the
    1024-instance batch, same shapes)."""
    cfg = dict(synth.CONFIG_DFT_C64_BATCH)
    cfg["B"] = 4
    inst = synth.make_batch(**cfg)
    plan = binding.Plan(inst["N"], inst["omega"], "dft", "fp32")
    res = plan.omp(torch.from_numpy(inst["Y"]).cuda(), inst["K"], path=path)
    assert plan.device_error() == 0
    check_omp(inst, res, "fp32", False)


def test_omp_edge_cases():
    kind, prec, N, M = "dft", "fp64", 64, 20
    om = omega_for(N, M, 1)
    plan = binding.Plan(N, om, kind, prec)
    # y = 0 halts before the first iteration
    y = torch.zeros(2, M, dtype=torch.complex128, device="cuda")
    x, supp, iters, rn = plan.omp(y, 5)
    assert iters.cpu().tolist() == [0, 0] and (supp.cpu().numpy() == -1).all() and (rn.cpu().numpy() == 0).all()
    # K = 0
    inst = synth.make_batch(kind, N, M, 3, 2, prec=prec, seed=4)
    x, supp, iters, rn = plan.omp(torch.from_numpy(inst["Y"]).cuda(), 0)
    assert iters.cpu().tolist() == [0, 0]
    # batch = 0
    x, supp, iters, rn = plan.omp(torch.zeros(0, M, dtype=torch.complex128, device="cuda"), 3)
    assert iters.numel() == 0


def test_omp_full_sampling_closed_form():
    """Omega = [0, N): selection in decreasing |x| and exact x."""
    N, K = 256, 10
    om = np.arange(N, dtype=np.int32)
    rng = np.random.default_rng(5)
    for kind in ("wht", "dft"):
        lam = synth.draw_support(N, K, rng)
        vals = synth.draw_values(K, kind, "gauss", rng)
        y = synth.measure(kind, N, om, lam, vals)[None]
        plan = binding.Plan(N, om, kind, "fp64")
        x, supp, iters, _ = plan.omp(torch.from_numpy(y).cuda(), K, path="fast")
        order = lam[np.argsort(-np.abs(vals), kind="stable")]
        assert supp[0].cpu().numpy().tolist() == order.tolist()
        xs = dict(zip(lam.tolist(), vals.tolist()))
        assert np.allclose(x[0].cpu().numpy(), [xs[j] for j in order.tolist()], atol=1e-12)


def test_omp_many_instances_per_cta():
    """More instances than resident CTAs: the persistent loop reuses smem and
    workspace; results must not depend on which CTA took an instance."""
    inst = synth.make_batch("wht", 256, 64, 6, 3000, prec="fp32", seed=8)
    plan = binding.Plan(256, inst["omega"], "wht", "fp32")
    y = torch.from_numpy(inst["Y"]).cuda()
    a = [t.cpu().numpy() for t in plan.omp(y, 6, path="hybrid")]
    b = [t.cpu().numpy() for t in plan.omp(y.flip(0).contiguous(), 6, path="hybrid")]
    assert np.array_equal(a[1], b[1][::-1]) and np.array_equal(a[0], b[0][::-1])
    check_omp({**inst, "B": 3}, [torch.from_numpy(v[:3]) for v in a], "fp32", True)


def test_omp_tie_break_by_hand():
    """Columns 1 and 3 coincide on Omega = {0, 1} (N = 4, WHT): the tie goes
    to the lower index (hand-derived fixture)."""
    plan = binding.Plan(4, np.array([0, 1], np.int32), "wht", "fp64")
    y = torch.tensor([[1.5, -1.5]], dtype=torch.float64, device="cuda")
    for path in ("fast", "conv"):
        x, supp, iters, _ = plan.omp(y, 2, path=path)
        assert supp[0].cpu().tolist()[:1] == [1] and int(iters[0]) == 1
        assert abs(float(x[0, 0]) - 3.0) < 1e-14
