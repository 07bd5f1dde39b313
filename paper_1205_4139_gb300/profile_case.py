"""One cs_omp launch per correlation path on a small batch of the
partial-DFT complex64 workload (N=4096, M=1024, K=64, 40 dB), then one
cs_correlate launch: the case the committed ncu summaries capture.  With
`single`, the same launches on the one partial-WHT FP64 instance (N=1024,
M=256, K=16, noiseless) of the latency measurement.

  python -m paper_1205_4139_gb300.profile_case [batch]
  python -m paper_1205_4139_gb300.profile_case 1 single
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    import torch

    import synth
    from paper_1205_4139_gb300 import binding

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
