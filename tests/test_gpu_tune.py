"""The measured switch point (cs_plan_tune, Sec. IV's adaptive strategy with
the crossover measured): the tuner reports a point from its ladder, a later
cs_omp with t_switch < 0 uses it, and the hybrid run it selects gives the
oracle's supports like every other switch point."""
import numpy as np
import pytest

import synth
from oracle import matrices, omp as oomp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1205_4139_gb300 import binding  # noqa: E402


@pytest.mark.parametrize("kind,prec,N,M,K", [("dft", "fp32", 1024, 256, 24), ("wht", "fp64", 512, 160, 20)])
def test_tune_then_default_switch(kind, prec, N, M, K):
    inst = synth.make_batch(kind, N, M, K, 40, snr_db=None, dist="gauss", prec=prec, seed=7)
    plan = binding.Plan(N, inst["omega"], kind, prec)
    y = torch.from_numpy(inst["Y"]).cuda()
    assert plan.switch_point() == 64  # the GB300 crossover of one-CTA plans, before tuning
    t_best, curve = plan.tune(y, K, rel_tol=1e-6)
    assert plan.switch_point() == t_best
    assert t_best in curve and 1 in curve and K in curve
    assert plan.info()["t_switch_default"] in curve
    assert all(v > 0 for v in curve.values())
    assert curve[t_best] == min(curve.values())
    assert plan.device_error() == 0

    xa, sa, ia, ra = plan.omp(y, K, path="hybrid", t_switch=-1)
    xb, sb, ib, rb = plan.omp(y, K, path="hybrid", t_switch=t_best)
    torch.cuda.synchronize()
    assert torch.equal(sa, sb) and torch.equal(ia, ib)
    assert torch.equal(xa, xb) and torch.equal(ra, rb)

    # the tuned hybrid run selects the oracle's columns (instances without a
    # near tie, the rule every OMP parity test uses)
    Phi = matrices.sensing(kind, N, inst["omega"])
    supp = sa.cpu().numpy()
    checked = 0
    for b in range(0, 40, 3):
        ref = oomp.omp(Phi, inst["Y"][b].astype(np.complex128 if kind == "dft" else np.float64), K)
        if min(ref["gap"]) <= 1e-3:
            continue
        assert supp[b][: ref["iters"]].tolist() == list(ref["support"])
        checked += 1
    assert checked >= 5


def test_tune_rejects_bad_arguments():
    om = synth.draw_omega(256, 64, np.random.default_rng(1))
    plan = binding.Plan(256, om, "dft", "fp32")
    y = torch.zeros(4, 64, dtype=torch.complex64, device="cuda")
    with pytest.raises(binding.CsError):
        plan.tune(y, 0)
    with pytest.raises(binding.CsError):
        plan.tune(y, 65)


def test_untuned_large_plan_uses_measured_crossover():
    om = synth.draw_omega(1 << 16, 8192, np.random.default_rng(2))
    assert binding.Plan(1 << 16, om, "dft", "fp32").switch_point() == 128
    assert binding.Plan(1 << 14, om[om < (1 << 14)], "wht", "fp32").switch_point() == 160
