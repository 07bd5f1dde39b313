"""The conventional correlation of partial-WHT FP32 plans on the tensor
cores (plans created with CS_PLAN_TENSOR_CORES; cs_correlate:
h = A^H zf_Omega(r), Algorithm 1.1 step 2, the FHT of Sec. III-B) against the
FP64 oracle.

The radix-16 Hadamard stages run as tcgen05 MMAs on three BF16 parts of the
FP32 data (exact: +-1 times an exactly split value), accumulated in FP32, so
h carries FP32 accumulation error only: far inside the 2e-5 FP32 tolerance
(the tests ask for 1e-6).  Sizes cover one vector per CTA round (N = 4096),
many vectors per round (N = 16 .. 2048), the CUDA-core path above 4096, a ragged last round, the remainder
stage (log2 N mod 4 = 1, 2, 3), values over 12 orders of magnitude (the split
must keep every bit), exact ties of |h| (lowest j wins) and the status word.
"""
import numpy as np
import pytest

import synth
from oracle import matrices, omp as oomp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1205_4139_gb300 import binding  # noqa: E402


def rel_inf(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("N,M,B", [(16, 7, 1), (16, 16, 1000), (32, 11, 300), (64, 30, 257), (256, 100, 70),
                                   (512, 200, 33), (1024, 256, 17), (2048, 900, 9), (4096, 1024, 5),
                                   (8192, 2000, 3)])
def test_tc_correlate_matches_oracle(N, M, B):
    rng = np.random.default_rng(N + B)
    om = synth.draw_omega(N, M, rng)
    plan = binding.Plan(N, om, "wht", "fp32", tensor_cores=True)
    r = rng.standard_normal((B, M)).astype(np.float32)
    h, am = plan.correlate(torch.from_numpy(r).cuda())
    h, am = h.cpu().numpy(), am.cpu().numpy()
    Phi = matrices.sensing_rows("wht", N, om)
    for b in sorted({0, B // 2, B - 1}):
        want = oomp.correlate(Phi, r[b].astype(np.float64)).real
        assert rel_inf(h[b], want) < 1e-6, (b, rel_inf(h[b], want))
        j, gap = oomp.identify(want, [])
        if gap > 1e-3:
            assert am[b] == j
    assert plan.device_error() == 0


@pytest.mark.parametrize("N", [256, 4096])
def test_tc_split_keeps_every_bit(N):
    """A single nonzero x with 24 significant bits: h(j) = +-x / sqrt(N)
    exactly (sqrt(N) is a power of two here).  Each stage's split
    x = hi + mid + lo is exact and the products by +-1 are exact, so the
    tensor-core path returns it bit for bit; a two-part split would lose the
    last 8 bits (relative error up to 2^-17)."""
    rng = np.random.default_rng(N)
    B = 8
    pos = rng.integers(0, N, size=B)
    mant = 1.0 + (2 * rng.integers(0, 2 ** 22, size=B) + 1) * 2.0 ** -23  # 24 significant bits
    x = (mant * 2.0 ** rng.integers(-20, 20, size=B) * rng.choice([-1.0, 1.0], size=B)).astype(np.float32)
    assert np.array_equal(x.astype(np.float64), mant * np.abs(x) / mant * np.sign(x))  # exact in FP32
    r = np.zeros((B, N), np.float32)
    r[np.arange(B), pos] = x
    plan = binding.Plan(N, np.arange(N, dtype=np.int32), "wht", "fp32", tensor_cores=True)
    h, _ = plan.correlate(torch.from_numpy(r).cuda())
    h = h.cpu().numpy()
    j = np.arange(N)
    for b in range(B):
        sign = 1.0 - 2.0 * (np.bitwise_count(j & int(pos[b])) & 1)
        want = (sign * np.float64(x[b]) / np.sqrt(N)).astype(np.float32)
        assert np.array_equal(h[b], want), b


def test_tc_exact_ties_go_to_lowest_index():
    """Full sampling, r = two equal spikes: |h| is constant over j, every j
    ties, and the arg-max is j = 0."""
    N = 256
    plan = binding.Plan(N, np.arange(N, dtype=np.int32), "wht", "fp32", tensor_cores=True)
    r = np.zeros((3, N), np.float32)
    r[:, 5] = 1.0
    r[1, 9] = 2.0  # |h| takes two values; ties among the larger ones
    h, am = plan.correlate(torch.from_numpy(r).cuda())
    h, am = h.cpu().numpy(), am.cpu().numpy()
    assert am[0] == 0 and am[2] == 0
    a = h[1] ** 2
    assert am[1] == int(np.flatnonzero(a == a.max())[0])


def test_tc_argmax_only_and_empty_batch():
    N, M = 1024, 300
    om = synth.draw_omega(N, M, np.random.default_rng(3))
    plan = binding.Plan(N, om, "wht", "fp32", tensor_cores=True)
    r = torch.from_numpy(np.random.default_rng(4).standard_normal((40, M)).astype(np.float32)).cuda()
    h, am = plan.correlate(r)
    _, am2 = plan.correlate(r, want_h=False)
    assert torch.equal(am, am2)
    plan.correlate(torch.zeros(0, M, dtype=torch.float32, device="cuda"))
    assert plan.device_error() == 0


def test_tc_flag_only_on_wht_fp32():
    for kind, prec in (("dft", "fp32"), ("wht", "fp64")):
        with pytest.raises(binding.CsError):
            binding.Plan(64, np.arange(8, dtype=np.int32), kind, prec, tensor_cores=True)


def test_tc_equals_cuda_core_path_to_rounding():
    N, M, B = 4096, 1024, 64
    om = synth.draw_omega(N, M, np.random.default_rng(5))
    r = torch.from_numpy(np.random.default_rng(6).standard_normal((B, M)).astype(np.float32)).cuda()
    ht, at = binding.Plan(N, om, "wht", "fp32", tensor_cores=True).correlate(r)
    hc, ac = binding.Plan(N, om, "wht", "fp32").correlate(r)
    ht, hc = ht.cpu().numpy(), hc.cpu().numpy()
    assert np.max(np.abs(ht - hc)) <= 1e-6 * np.max(np.abs(hc))
