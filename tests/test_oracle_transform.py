"""Pins of the large-N oracle (transform-based Algorithm 1.1) against the
dense oracle and against what the mathematics fixes, CPU only."""
import numpy as np
import pytest

import synth
from oracle import kernelsum, matrices, omp as oomp, transform as tro

MODES = ["wht", "dft"]


@pytest.mark.parametrize("N", [1, 2, 4, 16, 256, 1024])
def test_fwht_is_sylvester(N):
    rng = np.random.default_rng(N)
    v = rng.standard_normal((3, N))
    H = matrices.hadamard(N) * np.sqrt(N)  # Kronecker construction, unnormalised
    assert np.allclose(tro.fwht(v), v @ H.T, atol=1e-10 * np.sqrt(N))


def test_fwht_involution_and_energy():
    rng = np.random.default_rng(3)
    v = rng.standard_normal(2048)
    w = tro.fwht(v)
    assert np.allclose(tro.fwht(w) / 2048, v, atol=1e-12)
    assert np.isclose(np.dot(w, w), 2048 * np.dot(v, v), rtol=1e-12)


@pytest.mark.parametrize("kind", MODES)
@pytest.mark.parametrize("N,M", [(64, 20), (1024, 300), (4096, 1024)])
def test_correlate_and_synthesize_match_dense(kind, N, M):
    rng = np.random.default_rng(N + M)
    om = synth.draw_omega(N, M, rng)
    Phi = matrices.sensing(kind, N, om) if N <= 1024 else matrices.sensing_rows(kind, N, om)
    r = rng.standard_normal(M) + (1j * rng.standard_normal(M) if kind == "dft" else 0)
    h = tro.correlate(kind, N, om, r)
    assert np.max(np.abs(h - Phi.conj().T @ r)) < 1e-12 * np.max(np.abs(h))
    supp = rng.choice(N, 9, replace=False)
    x = rng.standard_normal(9) + (1j * rng.standard_normal(9) if kind == "dft" else 0)
    a = tro.synthesize(kind, N, om, supp, x)
    assert np.max(np.abs(a - Phi[:, supp] @ x)) < 1e-12 * max(1.0, np.max(np.abs(a)))
    assert np.allclose(tro.columns(kind, N, om, supp), Phi[:, supp], atol=1e-14)


@pytest.mark.parametrize("kind", MODES)
def test_kernel_vector_matches_definition(kind):
    N, M = 512, 131
    om = synth.draw_omega(N, M, np.random.default_rng(5))
    c = tro.kernel_vector(kind, N, om)
    assert np.max(np.abs(c - kernelsum.kernel_vector(kind, N, om))) < 1e-14
    assert np.isclose(c[0].real, M / N, rtol=0, atol=1e-15)


@pytest.mark.parametrize("kind", MODES)
def test_full_sampling_kernel_is_delta(kind):
    N = 1 << 14
    c = tro.kernel_vector(kind, N, np.arange(N))
    e0 = np.zeros(N)
    e0[0] = 1.0
    assert np.max(np.abs(c - e0)) < 1e-12


@pytest.mark.parametrize("kind", MODES)
@pytest.mark.parametrize("N,M,K,snr", [(1024, 256, 16, None), (2048, 400, 24, 30), (4096, 1024, 40, 40)])
def test_omp_matches_dense_oracle(kind, N, M, K, snr):
    inst = synth.make_batch(kind, N, M, K, 3, snr_db=snr, prec="fp64", seed=11)
    Phi = matrices.sensing_rows(kind, N, inst["omega"])
    for b in range(3):
        y = inst["Y"][b]
        a = oomp.omp(Phi, y, K)
        t = tro.omp(kind, N, inst["omega"], y, K)
        assert t["iters"] == a["iters"] and t["halt"] == a["halt"]
        assert t["support"] == a["support"]
        assert np.max(np.abs(np.asarray(t["x"]) - np.asarray(a["x"]))) < 1e-10 * np.max(np.abs(a["x"]))
        assert np.allclose(t["resnorm"], a["resnorm"], rtol=1e-9, atol=1e-12 * a["ynorm"])


@pytest.mark.parametrize("kind", MODES)
def test_omp_large_noiseless_recovery(kind):
    N, M, K = 1 << 14, 2048, 32
    inst = synth.make_batch(kind, N, M, K, 1, snr_db=None, prec="fp64", seed=2)
    t = tro.omp(kind, N, inst["omega"], inst["Y"][0], K)
    assert sorted(t["support"]) == sorted(inst["support"][0].tolist())
    order = np.argsort(t["support"])
    want = inst["values"][0][np.argsort(inst["support"][0])]
    assert np.max(np.abs(np.asarray(t["x"])[order] - want)) < 1e-10
    # orthogonality of the final residual to the chosen columns (step 6)
    r = inst["Y"][0] - tro.synthesize(kind, N, inst["omega"], t["support"], t["x"])
    h = tro.correlate(kind, N, inst["omega"], r)
    assert np.max(np.abs(h[t["support"]])) < 1e-10


@pytest.mark.parametrize("kind", MODES)
@pytest.mark.parametrize("algo", ["sp", "cosamp"])
@pytest.mark.parametrize("N,M,K,snr", [(512, 160, 8, None), (1024, 300, 12, 30)])
def test_pursuits_match_dense_oracle(kind, algo, N, M, K, snr):
    from oracle import pursuits
    inst = synth.make_batch(kind, N, M, K, 2, snr_db=snr, prec="fp64", seed=N + K)
    Phi = matrices.sensing(kind, N, inst["omega"])
    for b in range(2):
        y = inst["Y"][b]
        if algo == "sp":
            a = pursuits.subspace_pursuit(Phi, y, K)
            t = tro.subspace_pursuit(kind, N, inst["omega"], y, K)
        else:
            a = pursuits.cosamp(Phi, y, K)
            t = tro.cosamp(kind, N, inst["omega"], y, K)
        assert t["iters"] == a["iters"]
        assert list(t["support"]) == list(a["support"])
        assert np.max(np.abs(np.asarray(t["x"]) - np.asarray(a["x"]))) < 1e-10
        assert np.allclose(t["resnorm"], a["resnorm"], rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("kind", MODES)
@pytest.mark.parametrize("algo", ["sp", "cosamp"])
def test_large_pursuits_recover_noiseless(kind, algo):
    N, M, K = 1 << 14, 2048, 16
    inst = synth.make_batch(kind, N, M, K, 1, snr_db=None, prec="fp64", seed=31)
    f = tro.subspace_pursuit if algo == "sp" else tro.cosamp
    r = f(kind, N, inst["omega"], inst["Y"][0], K)
    assert sorted(r["support"].tolist()) == sorted(inst["support"][0].tolist())
