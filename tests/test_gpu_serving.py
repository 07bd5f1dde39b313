"""The request runtime on the GPU: jobs of mixed N (one-CTA and large
plans), kinds, precisions and algorithms give the same results in the mix
(several workers, a memory budget that makes jobs queue) as each job solved
alone through the plan API; a job larger than the budget is refused."""
import numpy as np
import pytest

import synth
from oracle import transform as tro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1205_4139_gb300 import binding  # noqa: E402

# (kind, prec, N, M, K, algo, snr)
JOBS = [
    ("wht", "fp64", 1024, 256, 16, "omp", None),
    ("dft", "fp32", 4096, 1024, 32, "omp", 40),
    ("dft", "fp32", 1 << 14, 2048, 24, "omp", None),
    ("wht", "fp32", 1 << 15, 4096, 40, "omp", 30),
    ("dft", "fp64", 1 << 14, 1500, 20, "omp", None),
    ("dft", "fp32", 2048, 512, 8, "cosamp", None),
    ("wht", "fp64", 1024, 300, 8, "sp", None),
    ("dft", "fp32", 1 << 16, 8192, 64, "omp", 40),
    ("wht", "fp64", 1 << 14, 2048, 12, "omp", None),
    ("dft", "fp32", 512, 128, 6, "cosamp", 40),
]


def make_jobs():
    out = []
    for i, (kind, prec, N, M, K, algo, snr) in enumerate(JOBS):
        inst = synth.make_batch(kind, N, M, K, 1, snr_db=snr, prec=prec, seed=100 + i)
        out.append((kind, prec, N, K, algo, inst))
    return out


def alone(job):
    kind, prec, N, K, algo, inst = job
    plan = binding.Plan(N, inst["omega"], kind, prec)
    y = torch.from_numpy(inst["Y"]).cuda()
    if algo == "omp":
        x, supp, it, rn = plan.omp(y, K)
    else:
        x, supp, it, rn = plan.pursuit(algo, y, K, path="hybrid")
    torch.cuda.synchronize()
    return x.cpu().numpy()[0], supp.cpu().numpy()[0], int(it.item()), float(rn.item())


@pytest.fixture(scope="module")
def jobs():
    return make_jobs()


@pytest.fixture(scope="module")
def reference(jobs):
    return [alone(j) for j in jobs]


@pytest.mark.parametrize("workers,budget_scale", [(1, 100.0), (4, 100.0), (4, 1.6)])
def test_mix_equals_alone(jobs, reference, workers, budget_scale):
    # footprints are reported back; a first pass with a large budget learns them
    srv = binding.Server(workers=workers, budget_bytes=8 << 30)
    for kind, prec, N, K, algo, inst in jobs:
        srv.submit(kind, prec, N, inst["omega"], inst["Y"][0], K, algo=algo)
    first = srv.wait_all()
    srv.close()
    biggest = max(r["footprint_bytes"] for r in first)
    budget = int(biggest * budget_scale) if budget_scale < 10 else 8 << 30
    srv = binding.Server(workers=workers, budget_bytes=budget)
    tickets = [srv.submit(kind, prec, N, inst["omega"], inst["Y"][0], K, algo=algo)
               for kind, prec, N, K, algo, inst in jobs]
    res = {r["ticket"]: r for r in srv.wait_all()}
    srv.close()
    for t, ref in zip(tickets, reference):
        r = res[t]
        assert r["status"] == 0 and r["device_error"] == 0
        x0, s0, it0, rn0 = ref
        assert r["iters"] == it0 and r["resnorm"] == rn0
        assert np.array_equal(r["supp"], s0)
        assert np.array_equal(r["x"], x0)
        assert r["t_submit_us"] <= r["t_admit_us"] <= r["t_done_us"]


def test_overlap_and_budget_respected(jobs):
    """With 4 workers and room for every job, some jobs run at the same time
    (their admit-to-done intervals overlap); with a budget of one biggest job
    plus a little, the summed footprint of overlapping jobs stays in budget."""
    srv = binding.Server(workers=4, budget_bytes=8 << 30)
    for kind, prec, N, K, algo, inst in jobs:
        srv.submit(kind, prec, N, inst["omega"], inst["Y"][0], K, algo=algo)
    res = srv.wait_all()
    srv.close()
    iv = sorted((r["t_admit_us"], r["t_done_us"]) for r in res)
    assert any(iv[i + 1][0] < iv[i][1] for i in range(len(iv) - 1))

    budget = int(max(r["footprint_bytes"] for r in res) * 1.2)
    srv = binding.Server(workers=4, budget_bytes=budget)
    for kind, prec, N, K, algo, inst in jobs:
        srv.submit(kind, prec, N, inst["omega"], inst["Y"][0], K, algo=algo)
    res = srv.wait_all()
    srv.close()
    events = sorted([(r["t_admit_us"], r["footprint_bytes"]) for r in res] +
                    [(r["t_done_us"], -r["footprint_bytes"]) for r in res], key=lambda e: (e[0], e[1]))
    use = 0
    for _, d in events:
        use += d
        assert use <= budget


def test_supports_match_oracle_on_noiseless_large_jobs(jobs):
    srv = binding.Server(workers=3, budget_bytes=8 << 30)
    picked = [j for j in jobs if j[4] == "omp" and j[2] >= (1 << 14) and j[5]["prec"] == "fp64"]
    tickets = [srv.submit(kind, prec, N, inst["omega"], inst["Y"][0], K) for kind, prec, N, K, algo, inst in picked]
    res = {r["ticket"]: r for r in srv.wait_all()}
    srv.close()
    for t, (kind, prec, N, K, algo, inst) in zip(tickets, picked):
        ref = tro.omp(kind, N, inst["omega"], inst["Y"][0].astype(np.complex128 if kind == "dft" else np.float64), K)
        upto = next((i for i, g in enumerate(ref["gap"]) if g <= 1e-3), len(ref["gap"]))
        assert res[t]["supp"][:upto].tolist() == ref["support"][:upto]


def test_refusals():
    srv = binding.Server(workers=2, budget_bytes=1 << 20)
    inst = synth.make_batch("dft", 1 << 16, 8192, 16, 1, prec="fp32", seed=1)
    with pytest.raises(binding.CsError):  # footprint beyond the whole budget
        srv.submit("dft", "fp32", 1 << 16, inst["omega"], inst["Y"][0], 16)
    with pytest.raises(binding.CsError):  # K > M
        srv.submit("wht", "fp64", 64, np.arange(8), np.ones(8), 9)
    with pytest.raises(binding.CsError):  # CoSaMP beyond K = 128
        srv.submit("dft", "fp32", 1 << 16, inst["omega"], inst["Y"][0], 200, algo="cosamp")
    srv.close()


def test_concurrent_small_plans_with_different_shared_memory():
    """Many one-CTA jobs whose kernels need different amounts of shared
    memory (N 4096 / 8192, K 8 .. 256, both kinds) on 8 workers: every job
    succeeds and equals its solve alone (the per-kernel shared-memory limit
    is only ever raised, so concurrent launches never see it lowered)."""
    rng = np.random.default_rng(21)
    specs = []
    for i in range(48):
        N = int(rng.choice([4096, 8192]))
        M = N // int(rng.choice([4, 8]))
        specs.append(("dft" if i % 2 else "wht", N, M, int(rng.integers(8, 257))))
    insts = [synth.make_batch(k, N, M, K, 1, snr_db=None, prec="fp32", seed=500 + i)
             for i, (k, N, M, K) in enumerate(specs)]
    srv = binding.Server(workers=8, budget_bytes=8 << 30)
    tickets = [srv.submit(k, "fp32", N, inst["omega"], inst["Y"][0], K)
               for (k, N, M, K), inst in zip(specs, insts)]
    res = {r["ticket"]: r for r in srv.wait_all()}
    srv.close()
    assert all(res[t]["status"] == 0 and res[t]["device_error"] == 0 for t in tickets)
    for i in (0, 7, 19, 33):
        k, N, M, K = specs[i]
        x0, s0, it0, rn0 = alone((k, "fp32", N, K, "omp", insts[i]))
        r = res[tickets[i]]
        assert np.array_equal(r["supp"], s0) and np.array_equal(r["x"], x0) and r["iters"] == it0
