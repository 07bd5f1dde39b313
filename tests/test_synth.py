"""The seeded input generators shared by the oracle, the tests and the
benchmark: measurements follow the closed form of Phi's entries, batches are
reproducible from their seeds, and the serving and uneven-batch request
streams have the shapes their workloads state."""
import numpy as np
import pytest

import synth


@pytest.mark.parametrize("kind", ["dft", "wht"])
@pytest.mark.parametrize("K", [3, 40])
def test_measure_is_the_column_sum(kind, K):
    """y = sum_k x_k Phi[:, lambda_k] with Phi's entries from their closed
    forms; the DFT's table lookup (used above 8 atoms) gives the same bits as
    evaluating every column."""
    N, M = 1 << 12, 700
    rng = np.random.default_rng(K)
    omega = np.sort(rng.choice(N, M, replace=False)).astype(np.int32)
    sup = rng.choice(N, K, replace=False)
    x = rng.standard_normal(K) + (1j * rng.standard_normal(K) if kind == "dft" else 0.0)
    y = synth.measure(kind, N, omega, sup, x)
    ref = np.zeros(M, dtype=y.dtype)
    for k, v in zip(sup.tolist(), x.tolist()):
        ref += v * synth.sensing_column(kind, N, omega, k)
    assert np.array_equal(y, ref)
    # and against the definition written out: (-1)^popcount / sqrt(N), or
    # exp(-2 pi i m k / N) / sqrt(N)
    om = omega.astype(np.int64)[:, None]
    kk = sup.astype(np.int64)[None, :]
    if kind == "wht":
        A = (1.0 - 2.0 * (np.bitwise_count(om & kk) & 1)) / np.sqrt(N)
    else:
        A = np.exp(-2j * np.pi * ((om * kk) % N) / N) / np.sqrt(N)  # the phase reduced exactly first
    assert np.max(np.abs(y - A @ x)) < 1e-12 * np.max(np.abs(y))


def test_batches_reproducible_and_shared_omega():
    a = synth.make_batch("dft", 512, 128, 6, 3, snr_db=40.0, prec="fp32", seed=9)
    b = synth.make_batch("dft", 512, 128, 6, 3, snr_db=40.0, prec="fp32", seed=9)
    assert np.array_equal(a["Y"], b["Y"]) and np.array_equal(a["omega"], b["omega"])
    assert a["Y"].dtype == np.complex64 and a["omega"].dtype == np.int32
    assert np.all(np.diff(a["omega"]) > 0)
    for s in a["support"]:
        assert len(set(s.tolist())) == 6


def test_uneven_batch_shapes():
    specs = synth.uneven_batch(300, seed=1)
    for sp in specs:
        assert 1 << 12 <= sp["N"] <= 1 << 16 and sp["N"] & (sp["N"] - 1) == 0
        assert sp["M"] in (sp["N"] // 4, sp["N"] // 8)
        assert 8 <= sp["K"] <= 256 and sp["kind"] in ("wht", "dft") and sp["dist"] in ("gauss", "rademacher")


def test_serving_cosamp_k_within_its_least_squares():
    """CoSaMP requests keep 3K <= M (its least squares run on up to 3K of the
    M rows); OMP requests keep K <= M."""
    for r in synth.serving_requests(500, seed=2):
        assert r["K"] <= r["M"]
        if r["algo"] == "cosamp":
            assert 3 * r["K"] <= r["M"]
