"""cs_omp_batched through the C ABI: OMP (Algorithm 1.1) on an uneven batch
of instances that each have their own plan (own Omega, N up to 2^16, M,
kind, precision) and their own K, one persistent kernel per element type.

* N <= 8192: bit for bit the results of cs_omp on the instance's plan (the
  same blocks in the same arithmetic order).
* N > 8192: the one-CTA radix-16 chains on global-memory buffers; parity
  with the FP64 transform oracle under the large-plan tolerances (supports
  exact up to the first oracle top-two gap <= 1e-3, x within 1e-10 / 1e-4
  relative in noiseless cases, ||r|| / ||y||), and agreement with cs_omp's
  four-step path.
* N > 2^16: cs_omp's large-plan path, bit for bit.
* the three correlation paths agree; edge cases (K = 0, y = 0, a plan shared
  by several instances, K = M, K = 1024, N = 2^16); refusals.
"""
import numpy as np
import pytest

import synth
from omp_checks import halting_ambiguous, resnorm_tol
from oracle import transform as tro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1205_4139_gb300 import binding  # noqa: E402

TOL_X = {"fp64": 1e-10, "fp32": 1e-4}


def wt(kind):
    return np.complex128 if kind == "dft" else np.float64


def build(specs, seed):
    """specs: (kind, prec, N, M, K, snr) -> (plans, ys, Ks, instances)."""
    plans, ys, Ks, insts = [], [], [], []
    for i, (kind, prec, N, M, K, snr) in enumerate(specs):
        inst = synth.make_batch(kind, N, M, K, 1, snr_db=snr, prec=prec, seed=seed * 1000 + i)
        plans.append(binding.Plan(N, inst["omega"], kind, prec))
        ys.append(torch.from_numpy(inst["Y"][0]).cuda())
        Ks.append(K)
        insts.append(inst)
    return plans, ys, Ks, insts


def check_against_oracle(inst, x, supp, iters, res, noiseless):
    """One instance against the transform oracle; returns whether the whole
    run was compared (no near tie)."""
    kind, prec, N, K = inst["kind"], inst["prec"], inst["N"], inst["K"]
    ref = tro.omp(kind, N, inst["omega"], inst["Y"][0].astype(wt(kind)), K)
    upto = next((t for t, g in enumerate(ref["gap"]) if g <= 1e-3), len(ref["gap"]))
    assert supp[:upto].tolist() == ref["support"][:upto]
    if upto < len(ref["gap"]):
        return False
    assert iters == ref["iters"] or halting_ambiguous(ref, prec)
    if noiseless and ref["halt"] != "dependent":
        xr = np.asarray(ref["x"])
        n = min(iters, len(xr))
        assert np.max(np.abs(x[:n] - xr[:n])) < TOL_X[prec] * np.max(np.abs(xr))
    if ref["resnorm"]:
        rr = ref["resnorm"][-1] / ref["ynorm"]
        assert abs(res - rr) <= resnorm_tol(rr, prec), (res, rr)
    return True


def small_specs(seed, n=24):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        kind = ("wht", "dft")[i % 2]
        prec = ("fp32", "fp64")[(i // 2) % 2]
        N = 1 << int(rng.integers(6, 14))
        M = N // int(rng.choice([4, 8]))
        K = int(rng.integers(1, min(M, 80) + 1))
        out.append((kind, prec, N, M, K, None if i % 3 else 40))
    return out


@pytest.mark.parametrize("path", ["fast", "conv", "hybrid"])
def test_small_plans_equal_cs_omp(path):
    plans, ys, Ks, _ = build(small_specs(3), 3)
    bt = binding.omp_batched(plans, ys, Ks, path=path)
    torch.cuda.synchronize()
    for b, (p, y, K) in enumerate(zip(plans, ys, Ks)):
        x, s, it, rn = p.omp(y[None], K, path=path)
        torch.cuda.synchronize()
        assert torch.equal(bt.supp[b], s[0]), b
        assert torch.equal(bt.x[b], x[0]), b
        assert int(bt.iters[b]) == int(it[0]) and float(bt.resnorm[b]) == float(rn[0])
    assert plans[0].device_error() == 0


BIG = [("dft", "fp32", 1 << 14, 2048, 24, None), ("wht", "fp32", 1 << 15, 4096, 40, None),
       ("dft", "fp64", 1 << 16, 8192, 30, None), ("wht", "fp64", 1 << 14, 1500, 20, 40),
       ("dft", "fp32", 1 << 16, 6000, 48, 40), ("wht", "fp32", 1 << 16, 8192, 64, None)]


@pytest.mark.parametrize("path", ["fast", "conv", "hybrid"])
def test_big_plans_match_oracle(path):
    plans, ys, Ks, insts = build(BIG, 5)
    bt = binding.omp_batched(plans, ys, Ks, path=path, t_switch=9)
    torch.cuda.synchronize()
    compared = 0
    for b, inst in enumerate(insts):
        compared += check_against_oracle(inst, bt.x[b].cpu().numpy(), bt.supp[b].cpu().numpy(),
                                         int(bt.iters[b]), float(bt.resnorm[b]), BIG[b][5] is None)
    assert compared >= 3
    assert plans[0].device_error() == 0


def test_big_plans_agree_with_four_step_path():
    plans, ys, Ks, insts = build(BIG, 6)
    bt = binding.omp_batched(plans, ys, Ks)
    torch.cuda.synchronize()
    for b, (p, y, K, inst) in enumerate(zip(plans, ys, Ks, insts)):
        x, s, it, rn = p.omp(y[None], K)
        ref = tro.omp(inst["kind"], inst["N"], inst["omega"], inst["Y"][0].astype(wt(inst["kind"])), K)
        upto = next((t for t, g in enumerate(ref["gap"]) if g <= 1e-3), len(ref["gap"]))
        assert bt.supp[b].cpu().numpy()[:upto].tolist() == s[0].cpu().numpy()[:upto].tolist()
        if upto == len(ref["gap"]) and int(it[0]) == int(bt.iters[b]):
            xa, xb = bt.x[b].cpu().numpy(), x[0].cpu().numpy()
            assert np.max(np.abs(xa - xb)) <= 2 * TOL_X[inst["prec"]] * max(np.max(np.abs(xb)), 1e-30)


def test_uneven_mix_small_exact_big_oracle():
    """The uneven workload's recipe (N = 2^12 .. 2^16, M = N/4 or N/8,
    WHT FP32 / DFT complex64, per-instance Omega, noiseless) at K <= 40:
    one-CTA instances equal cs_omp bit for bit, the others match the oracle."""
    specs = synth.uneven_batch(20, seed=11, k_hi=40)
    plans, ys, Ks, insts = [], [], [], []
    for sp in specs:
        om, yv = synth.uneven_instance(sp)
        plans.append(binding.Plan(sp["N"], om, sp["kind"], "fp32"))
        ys.append(torch.from_numpy(yv).cuda())
        Ks.append(sp["K"])
        insts.append({"kind": sp["kind"], "prec": "fp32", "N": sp["N"], "K": sp["K"], "omega": om, "Y": yv[None]})
    bt = binding.omp_batched(plans, ys, Ks)
    torch.cuda.synchronize()
    for b, (p, y, K) in enumerate(zip(plans, ys, Ks)):
        if p.N <= 8192:
            x, s, it, rn = p.omp(y[None], K)
            assert torch.equal(bt.supp[b], s[0]) and torch.equal(bt.x[b], x[0])
        else:
            check_against_oracle(insts[b], bt.x[b].cpu().numpy(), bt.supp[b].cpu().numpy(), int(bt.iters[b]),
                                 float(bt.resnorm[b]), True)


def test_edge_cases():
    specs = [("dft", "fp32", 1 << 14, 1024, 12, None), ("wht", "fp32", 4096, 512, 12, None),
             ("wht", "fp64", 64, 16, 16, None), ("dft", "fp64", 1 << 15, 2048, 10, None)]
    plans, ys, Ks, insts = build(specs, 8)
    # K = 0 on one instance, y = 0 on another, K = M on a third, one plan used twice
    Ks[1] = 0
    ys[3] = torch.zeros_like(ys[3])
    plans.append(plans[0])
    ys.append(ys[0] * 2)
    Ks.append(12)
    bt = binding.omp_batched(plans, ys, Ks)
    torch.cuda.synchronize()
    it = bt.iters.cpu().numpy()
    assert it[1] == 0 and bt.supp[1].numel() == 0
    assert it[3] == 0 and float(bt.resnorm[3]) == 0.0 and (bt.supp[3].cpu().numpy() == -1).all()
    assert sorted(bt.supp[0].cpu().numpy().tolist()) == sorted(insts[0]["support"][0].tolist())
    # y scaled by 2 on the same plan: the same support, x doubled
    assert torch.equal(bt.supp[4], bt.supp[0])
    assert torch.allclose(bt.x[4], 2 * bt.x[0], rtol=1e-5, atol=0)
    assert it[2] <= 16
    check_against_oracle(insts[2], bt.x[2].cpu().numpy(), bt.supp[2].cpu().numpy(), int(it[2]),
                         float(bt.resnorm[2]), True)
    # a single instance, and an empty batch
    one = binding.omp_batched(plans[:1], ys[:1], Ks[:1])
    torch.cuda.synchronize()
    assert torch.equal(one.supp[0], bt.supp[0])
    binding.omp_batched([], [], [])
    assert plans[0].device_error() == 0


def test_largest_sizes_by_properties():
    """N = 2^16 with K = 1024 (both limits): distinct columns, a residual
    orthogonal to them, and the reported residual norm (FP64 plan)."""
    N, M, K = 1 << 16, 4096, 1024
    inst = synth.make_batch("dft", N, M, 900, 1, snr_db=30, prec="fp64", seed=77)
    plan = binding.Plan(N, inst["omega"], "dft", "fp64")
    y = torch.from_numpy(inst["Y"][0]).cuda()
    bt = binding.omp_batched([plan], [y], [K])
    torch.cuda.synchronize()
    n = int(bt.iters[0])
    s = bt.supp[0].cpu().numpy()[:n]
    x = bt.x[0].cpu().numpy()[:n]
    assert n == K and len(set(s.tolist())) == n
    yv = inst["Y"][0]
    r = yv - tro.synthesize("dft", N, inst["omega"], s, x)
    h = tro.correlate("dft", N, inst["omega"], r)
    assert np.max(np.abs(h[s])) < 1e-8 * np.linalg.norm(yv)
    assert abs(float(bt.resnorm[0]) - np.linalg.norm(r) / np.linalg.norm(yv)) < 1e-7
    assert plan.device_error() == 0


def test_large_plans_ride_along():
    """Instances with N > 2^16 (the large-plan path, on library streams)
    beside one-CTA and global-memory ones: each equals cs_omp on its plan bit
    for bit, also when its plan is used twice in the call."""
    specs = [("dft", "fp32", 1 << 17, 8192, 40, None), ("wht", "fp64", 1 << 18, 9000, 24, 40),
             ("dft", "fp32", 2048, 512, 20, None), ("wht", "fp32", 1 << 15, 4096, 30, None)]
    plans, ys, Ks, insts = build(specs, 12)
    plans.append(plans[0])
    ys.append(ys[0] * 0.5)
    Ks.append(17)
    bt = binding.omp_batched(plans, ys, Ks)
    torch.cuda.synchronize()
    for b in (0, 1, 2, 4):
        x, s, it, rn = plans[b].omp(ys[b][None], Ks[b])
        torch.cuda.synchronize()
        assert torch.equal(bt.supp[b], s[0]) and torch.equal(bt.x[b], x[0]), b
        assert int(bt.iters[b]) == int(it[0]) and float(bt.resnorm[b]) == float(rn[0])
    check_against_oracle(insts[3], bt.x[3].cpu().numpy(), bt.supp[3].cpu().numpy(), int(bt.iters[3]),
                         float(bt.resnorm[3]), True)
    assert all(p.device_error() == 0 for p in plans[:4])


def test_refusals():
    rng = np.random.default_rng(1)
    om = synth.draw_omega(1 << 17, 5000, rng)
    big = binding.Plan(1 << 17, om, "dft", "fp32")
    y = torch.zeros(5000, dtype=torch.complex64, device="cuda")
    with pytest.raises(binding.CsError):  # K above 4096 for N > 2^16
        binding.omp_batched([big], [y], [4097])
    om2 = synth.draw_omega(1 << 14, 2048, rng)
    half = binding.Plan(1 << 14, om2, "dft", "fp32", c_storage="half")
    y2 = torch.zeros(2048, dtype=torch.complex64, device="cuda")
    with pytest.raises(binding.CsError):  # c not fully stored
        binding.omp_batched([half], [y2], [4])
    ok = binding.Plan(1 << 14, om2, "dft", "fp32")
    with pytest.raises(binding.CsError):  # K > 1024
        binding.omp_batched([ok], [y2], [1025])
    small = binding.Plan(64, np.arange(8), "wht", "fp64")
    with pytest.raises(binding.CsError):  # K > M
        binding.omp_batched([small], [torch.zeros(8, dtype=torch.float64, device="cuda")], [9])
    with pytest.raises(ValueError):  # y of the wrong length
        binding.omp_batched([small], [torch.zeros(7, dtype=torch.float64, device="cuda")], [2])


def test_batch_tuner_shapes_and_results():
    """cs_omp_batched_tune on a mix of residences and element types: one
    record per launch group present, shapes within their candidate sets, and
    cs_omp_batched with the stored shapes still matches the oracle (supports
    to the first near tie, noiseless x); count = 0 forgets the shapes."""
    specs = [("wht", "fp32", 4096, 1024, 20, None), ("dft", "fp32", 2048, 512, 24, None),
             ("dft", "fp32", 1 << 14, 2048, 30, None), ("wht", "fp32", 1 << 15, 4096, 24, None)] * 6
    plans, ys, Ks, insts = build(specs, 21)
    bt = binding.Batch(plans, ys, Ks)
    try:
        recs = binding.batch_tune(bt)
        assert sorted(r["group"] for r in recs) == ["dft fp32 global", "dft fp32 shared", "wht fp32 global",
                                                    "wht fp32 shared"]
        for r in recs:
            assert r["ctas_per_sm"] >= 0 and r["ms"] > 0
            assert r["t_switch"] in ((-1, 16, 64, 128) if r["group"].endswith("global") else (-1, 32, 128))
        bt.run()
        torch.cuda.synchronize()
        compared = 0
        for b in range(len(specs)):
            compared += check_against_oracle(insts[b], bt.x[b].cpu().numpy(), bt.supp[b].cpu().numpy(),
                                             int(bt.iters[b]), float(bt.resnorm[b]), True)
        assert compared >= 8
        assert plans[0].device_error() == 0
    finally:
        binding.batch_untune()
    # forgotten: small instances equal cs_omp at the plan's switch point again
    bt.run()
    torch.cuda.synchronize()
    x, s, it, rn = plans[0].omp(ys[0][None], Ks[0])
    assert torch.equal(bt.supp[0], s[0]) and torch.equal(bt.x[0], x[0])
