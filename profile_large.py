"""One launch of each large-plan kernel on a partial-DFT complex64 workload
(N = 2^22, M = 2^19): cs_correlate on `batch` measurements (the four-step
transform passes), cs_correlate_fast with s = 64 atoms, and cs_omp with K = 8
by transforms on one measurement (residual and adjoint passes, the
least-squares kernel): the case the committed ncu summaries of the large path
capture.

  python profile_large.py [batch]
"""
import os
import sys

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    import numpy as np
    import torch

    import synth
    from paper_1205_4139_gb300 import binding

    B = int(sys.argv[1]) if len(sys.argv) > 1 else 4
    N, M = 1 << 22, 1 << 19
    inst = synth.make_batch("dft", N, M, 8, B, snr_db=30, prec="fp32", seed=5)
    plan = binding.Plan(N, inst["omega"], "dft", "fp32")
    y = torch.from_numpy(inst["Y"]).cuda()
    h, _ = plan.correlate(y)
    rng = np.random.default_rng(1)
    sp = torch.from_numpy(np.stack([rng.choice(N, 64, replace=False) for _ in range(B)]).astype(np.int32)).cuda()
    xs = torch.from_numpy((rng.standard_normal((B, 64)) + 1j * rng.standard_normal((B, 64))).astype(np.complex64)).cuda()
    plan.correlate_fast(h, sp, xs, want_h=False)
    plan.omp(y[:1].contiguous(), 8, path="conv")
    torch.cuda.synchronize()
    print("ok")


if __name__ == "__main__":
    main()
