"""Small batches run on one thread-block cluster per instance
(cs_omp_cluster.cu); larger batches on the persistent kernel (cs_omp.cu).
Both take the same steps with the same arithmetic, so an instance solved in a
small batch equals the same instance solved in a large batch bit for bit,
for every kind, precision and correlation path."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1205_4139_gb300 import binding  # noqa: E402

MODES = [("wht", "fp64"), ("wht", "fp32"), ("dft", "fp64"), ("dft", "fp32")]


@pytest.mark.parametrize("kind,prec", MODES)
@pytest.mark.parametrize("path", ["fast", "conv", "hybrid"])
@pytest.mark.parametrize("N,M,K,snr", [(1024, 256, 16, None), (4096, 1024, 64, 40), (256, 64, 20, 20)])
def test_cluster_equals_persistent(kind, prec, path, N, M, K, snr):
    inst = synth.make_batch(kind, N, M, K, 48, snr_db=snr, prec=prec, seed=N + K)
    plan = binding.Plan(N, inst["omega"], kind, prec)
    y = torch.from_numpy(inst["Y"]).cuda()
    big = plan.omp(y, K, path=path, t_switch=9)              # 48 instances: persistent kernel
    for lo, hi in ((0, 1), (5, 9), (29, 48)):  # 1, 4 and 19 instances: clusters
        small = plan.omp(y[lo:hi].contiguous(), K, path=path, t_switch=9)
        torch.cuda.synchronize()
        for u, v in zip(big, small):
            assert torch.equal(u[lo:hi], v), (lo, hi)
    assert plan.device_error() == 0


def test_cluster_zero_and_tiny():
    N, M, K = 64, 16, 5
    inst = synth.make_batch("dft", N, M, K, 3, snr_db=None, prec="fp32", seed=1)
    Y = inst["Y"].copy()
    Y[1] = 0
    plan = binding.Plan(N, inst["omega"], "dft", "fp32")
    x, s, it, rn = plan.omp(torch.from_numpy(Y).cuda(), K)
    it = it.cpu().numpy()
    assert it[1] == 0 and rn.cpu().numpy()[1] == 0.0 and (s.cpu().numpy()[1] == -1).all()
    assert sorted(s.cpu().numpy()[0].tolist()) == sorted(inst["support"][0].tolist())
    x0, s0, i0, r0 = plan.omp(torch.from_numpy(Y).cuda(), 0)
    assert (i0.cpu().numpy() == 0).all()
