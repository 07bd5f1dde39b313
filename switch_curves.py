"""Per-iteration cost of the two correlations on GB300 as the support grows
(the GPU analogue of the paper's Figs. 1-2, Sec. IV): for each N, OMP is
timed with K = k for a ladder of k on the kernel-sum path (FAST) and on the
transform path (CONV); the slope between consecutive k is the cost of one
iteration at t ~ k.  Prints one JSON line per (kind, precision, N).

  python switch_curves.py [logN ...]
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def curve(kind, prec, logN, ks, batch, reps=3):
    import torch

    import synth
    from paper_1205_4139_gb300 import binding

    N = 1 << logN
    M = N // 4
    K = max(ks)
    inst = synth.make_batch(kind, N, M, K, batch, snr_db=30, prec=prec, seed=logN)
    plan = binding.Plan(N, inst["omega"], kind, prec)
    y = torch.from_numpy(inst["Y"]).cuda()
    out = {}
    for path in ("fast", "conv"):
        times = []
        for k in ks:
            plan.omp(y, k, path=path, rel_tol=0.0)  # warm-up (workspace)
            torch.cuda.synchronize()
            best = None
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                plan.omp(y, k, path=path, rel_tol=0.0)
                e1.record()
                torch.cuda.synchronize()
                t = e0.elapsed_time(e1)
                best = t if best is None else min(best, t)
            times.append(best)
        # ms per iteration per instance between consecutive ladder points
        out[path] = {str(ks[i + 1]): (times[i + 1] - times[i]) / (ks[i + 1] - ks[i]) / batch
                     for i in range(len(ks) - 1)}
        out[path + "_total_ms"] = dict(zip(map(str, ks), times))
    return {"kind": kind, "prec": prec, "logN": logN, "M": M, "batch": batch, "per_iteration_ms": out}


def main():
    logs = [int(a) for a in sys.argv[1:]] or [10, 12, 13, 14, 16, 18, 20]
    for logN in logs:
        for kind, prec in (("dft", "fp32"), ("wht", "fp32")):
            if logN <= 13:
                ks, batch = [8, 16, 32, 64, 96, 128], 304
            else:
                ks, batch = [16, 64, 128, 256, 512], 1
            print(json.dumps(curve(kind, prec, logN, ks, batch)), flush=True)


if __name__ == "__main__":
    main()
