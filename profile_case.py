"""One cs_omp launch per correlation path on a small batch of the
partial-DFT complex64 workload (N=4096, M=1024, K=64, 40 dB), then one
cs_correlate launch: the case the committed ncu summaries capture.  With
`single`, the same launches on the one partial-WHT FP64 instance (N=1024,
M=256, K=16, noiseless) of the latency measurement.  With `uneven`, the
first `count` instances of one kind (wht / dft / all) and residence (small:
N <= 8192, big: larger N, all) of the 4096-instance uneven batch, in two
cs_omp_batched calls (the second is the one to capture).

  python profile_case.py [batch]
  python profile_case.py 1 single
  python profile_case.py uneven dft big 304
  python profile_case.py wht_tc 16384 4096

With `cosamp N K`, one CoSaMP solve on a partial-DFT complex64 instance
(M = N/8, noiseless, its least squares by cluster conjugate gradients):

  python profile_case.py cosamp 1048576 1024

With `sp batch`, subspace pursuit (K = 64, kernel sums) on the first
`batch` instances of the partial-DFT complex64 workload:

  python profile_case.py sp 304

With `wht_tc`, two cs_correlate calls on `batch` residuals of a partial-WHT
FP32 plan with N points and M = N/4 rows (the tensor-core Hadamard stages;
the second call is the one to capture).
"""
import os
import sys

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def uneven(kind, residence, count):
    import torch

    import synth
    from paper_1205_4139_gb300 import binding

    def keep(s):
        return (kind == "all" or s["kind"] == kind) and (residence == "all" or (s["N"] > 8192) == (residence == "big"))

    specs = [s for s in synth.uneven_batch(4096, seed=0) if keep(s)][:count]
    plans, ys = [], []
    for sp in specs:
        om, yv = synth.uneven_instance(sp)
        plans.append(binding.Plan(sp["N"], om, sp["kind"], "fp32"))
        ys.append(torch.from_numpy(yv).cuda())
    bt = binding.Batch(plans, ys, [sp["K"] for sp in specs])
    for _ in range(2):
        bt.run()
    torch.cuda.synchronize()
    assert plans[0].device_error() == 0
    print("ok", len(specs), int(bt.iters.sum()))


def main():
    import torch

    import synth
    from paper_1205_4139_gb300 import binding

    if len(sys.argv) > 1 and sys.argv[1] == "uneven":
        uneven(sys.argv[2], sys.argv[3], int(sys.argv[4]))
        return
    if len(sys.argv) > 1 and sys.argv[1] == "wht_tc":
        import numpy as np
        B, N = int(sys.argv[2]), int(sys.argv[3])
        plan = binding.Plan(N, synth.draw_omega(N, N // 4, np.random.default_rng(1)), "wht", "fp32", tensor_cores=True)
        r = torch.randn(B, N // 4, device="cuda")
        for _ in range(2):
            plan.correlate(r)
        torch.cuda.synchronize()
        assert plan.device_error() == 0
        print("ok")
        return
    if len(sys.argv) > 1 and sys.argv[1] == "cosamp":
        # one CoSaMP solve on a partial-DFT complex64 instance with N points,
        # M = N/8 rows, noiseless, K atoms (least squares by the cluster
        # conjugate gradients of cs_cg.cuh)
        N, K = int(sys.argv[2]), int(sys.argv[3])
        inst = synth.make_batch("dft", N, N // 8, K, 1, snr_db=None, prec="fp32", seed=5)
        plan = binding.Plan(N, inst["omega"], "dft", "fp32")
        x, s, it, rn = plan.pursuit("cosamp", torch.from_numpy(inst["Y"]).cuda(), K, path="hybrid")
        torch.cuda.synchronize()
        assert plan.device_error() == 0
        print("ok", int(it[0]))
        return
    if len(sys.argv) > 1 and sys.argv[1] == "sp":
        # subspace pursuit (kernel sums) on the first `batch` instances of the
        # partial-DFT complex64 workload, K = 64
        cfg = dict(synth.CONFIG_DFT_C64_BATCH)
        cfg["B"] = int(sys.argv[2])
        inst = synth.make_batch(**cfg)
        plan = binding.Plan(cfg["N"], inst["omega"], cfg["kind"], cfg["prec"])
        x, s, it, rn = plan.pursuit("sp", torch.from_numpy(inst["Y"]).cuda(), cfg["K"], path="fast")
        torch.cuda.synchronize()
        print("ok", float(it.float().mean()))
        return
    B = int(sys.argv[1]) if len(sys.argv) > 1 else 456
    single = len(sys.argv) > 2 and sys.argv[2] == "single"
    cfg = dict(synth.CONFIG_WHT_FP64_SINGLE if single else synth.CONFIG_DFT_C64_BATCH)
    cfg["B"] = B
    inst = synth.make_batch(**cfg)
    plan = binding.Plan(cfg["N"], inst["omega"], cfg["kind"], cfg["prec"])
    y = torch.from_numpy(inst["Y"]).cuda()
    for path in ("fast", "conv"):
        plan.omp(y, cfg["K"], path=path)
    plan.correlate(y, want_h=False)
    torch.cuda.synchronize()
    print("ok")


if __name__ == "__main__":
    main()
