"""Pins of the SP and CoSaMP oracles (recovery and invariants; the paper
prints no iterate of either algorithm)."""
import numpy as np
import pytest

import synth
from oracle import matrices, omp, pursuits

KINDS = ["wht", "dft"]


def test_top_k_tie_break_and_exclusion():
    v = np.array([1.0, -3.0, 3.0, 0.5, -3.0])
    assert pursuits.top_k(v, 2).tolist() == [1, 2]          # |3| three times: lowest indices win
    assert pursuits.top_k(v, 2, excluded=[1]).tolist() == [2, 4]
    assert pursuits.top_k(v, 9).tolist() == [0, 1, 2, 3, 4]


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("algo", ["sp", "cosamp"])
@pytest.mark.parametrize("seed", [0, 1])
def test_exact_noiseless_recovery(kind, algo, seed):
    rng = np.random.default_rng(300 + seed)
    N, M, K = 256, 128, 6
    om = synth.draw_omega(N, M, rng)
    lam = synth.draw_support(N, K, rng)
    vals = synth.draw_values(K, kind, "gauss", rng)
    y = synth.measure(kind, N, om, lam, vals)
    Phi = matrices.sensing(kind, N, om)
    res = pursuits.subspace_pursuit(Phi, y, K) if algo == "sp" else pursuits.cosamp(Phi, y, K)
    assert sorted(res["support"].tolist()) == sorted(lam.tolist())
    xs = dict(zip(lam.tolist(), vals.tolist()))
    assert np.allclose(res["x"], [xs[j] for j in res["support"].tolist()], atol=1e-10)
    assert res["resnorm"][-1] < 1e-10 * res["ynorm"]


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("algo", ["sp", "cosamp"])
def test_agree_with_omp_on_one_sparse(kind, algo):
    """K = 1: SP and OMP pick the largest correlation and solve the same
    one-column least squares; CoSaMP keeps the same column after pruning a
    two-column solve (its coefficient is that solve's, not OMP's)."""
    rng = np.random.default_rng(5)
    N, M = 128, 40
    om = synth.draw_omega(N, M, rng)
    Phi = matrices.sensing(kind, N, om)
    y = synth.measure(kind, N, om, synth.draw_support(N, 1, rng), synth.draw_values(1, kind, "gauss", rng))
    y = synth.add_noise(y, 30.0, rng)
    o = omp.omp(Phi, y, 1)
    r = pursuits.subspace_pursuit(Phi, y, 1) if algo == "sp" else pursuits.cosamp(Phi, y, 1, max_iter=1)
    assert r["support"].tolist() == o["support"]
    if algo == "sp":
        assert np.allclose(r["x"], o["x"], atol=1e-12)


@pytest.mark.parametrize("kind", KINDS)
def test_sp_invariants(kind):
    """|T| = K, x is the least-squares solution on T (residual orthogonal to
    Phi_T) and the accepted residual norms decrease."""
    rng = np.random.default_rng(9)
    N, M, K = 256, 90, 10
    om = synth.draw_omega(N, M, rng)
    Phi = matrices.sensing(kind, N, om)
    y = synth.add_noise(synth.measure(kind, N, om, synth.draw_support(N, K, rng),
                                      synth.draw_values(K, kind, "gauss", rng)), 15.0, rng)
    res = pursuits.subspace_pursuit(Phi, y, K)
    T = res["support"]
    assert len(T) == K and len(set(T.tolist())) == K
    r = y - Phi[:, T] @ res["x"]
    assert np.max(np.abs(Phi[:, T].conj().T @ r)) < 1e-12 * np.linalg.norm(y)
    assert np.all(np.diff(res["resnorm"]) < 0)


@pytest.mark.parametrize("kind", KINDS)
def test_cosamp_invariants(kind):
    rng = np.random.default_rng(10)
    N, M, K = 256, 100, 8
    om = synth.draw_omega(N, M, rng)
    Phi = matrices.sensing(kind, N, om)
    y = synth.add_noise(synth.measure(kind, N, om, synth.draw_support(N, K, rng),
                                      synth.draw_values(K, kind, "gauss", rng)), 20.0, rng)
    res = pursuits.cosamp(Phi, y, K)
    assert len(res["support"]) <= K
    assert np.all(np.diff(res["resnorm"]) < 0)
    # the pruned x is exactly a least-squares b restricted to its K largest entries:
    # re-running the last step from the previous iterate reproduces it
    assert np.isclose(res["resnorm"][-1], np.linalg.norm(y - Phi[:, res["support"]] @ res["x"]))


def test_zero_measurement():
    Phi = matrices.sensing("dft", 32, np.arange(10))
    for f in (pursuits.subspace_pursuit, pursuits.cosamp):
        r = f(Phi, np.zeros(10, complex), 3)
        assert r["iters"] == 0 and len(r["support"]) == 0
