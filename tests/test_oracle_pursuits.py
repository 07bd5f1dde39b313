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


# ------------------------------------------------ iterates derived by hand
import json  # noqa: E402
import os  # noqa: E402
from fractions import Fraction  # noqa: E402

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "pursuits_by_hand.json")))


def _fr(v):
    return float(Fraction(v[0], v[1]))


def _case(c):
    N, om = c["N"], np.array(c["omega"])
    Phi = matrices.sensing(c["kind"], N, om)
    xt = np.zeros(N)
    for j, v in c["x_true"].items():
        xt[int(j)] = _fr(v)
    return Phi, Phi @ xt


@pytest.mark.parametrize("case", GOLD["sp"], ids=lambda c: c["name"])
def test_sp_iterates_by_hand(case):
    Phi, y = _case(case)
    res = pursuits.subspace_pursuit(Phi, y, case["K"])
    assert res["T0"].tolist() == case["T0"]
    assert np.allclose(res["x0"], [_fr(v) for v in case["x0"]], atol=1e-13)
    assert np.isclose(res["resnorm"][0] ** 2, _fr(case["rn0_sq"]), atol=1e-13)
    assert len(res["trace"]) == len(case["trace"])
    for got, want in zip(res["trace"], case["trace"]):
        assert got["Tp"].tolist() == want["Tp"] and got["Tn"].tolist() == want["Tn"]
        assert np.allclose(got["b"], [_fr(v) for v in want["b"]], atol=1e-13)
        assert np.allclose(got["x"], [_fr(v) for v in want["x"]], atol=1e-13)
        assert np.isclose(got["rn"] ** 2, _fr(want["rn_sq"]), atol=1e-13)
        assert got["accepted"] == want["accepted"]
    assert res["support"].tolist() == case["support"] and res["iters"] == case["iters"]
    assert np.allclose(res["x"], [_fr(v) for v in case["x"]], atol=1e-13)


@pytest.mark.parametrize("case", GOLD["cosamp"], ids=lambda c: c["name"])
def test_cosamp_iterates_by_hand(case):
    Phi, y = _case(case)
    assert np.isclose(np.vdot(y, y).real, _fr(case["ynorm_sq"]))
    res = pursuits.cosamp(Phi, y, case["K"])
    assert len(res["trace"]) == len(case["trace"])
    for got, want in zip(res["trace"], case["trace"]):
        assert got["T"].tolist() == want["T"] and got["S"].tolist() == want["S"]
        assert np.allclose(got["b"], [_fr(v) for v in want["b"]], atol=1e-13)
        assert np.allclose(got["x"], [_fr(v) for v in want["x"]], atol=1e-13)
        assert np.isclose(got["rn"] ** 2, _fr(want["rn_sq"]), atol=1e-13)
        assert got["accepted"] == want["accepted"]
    assert res["support"].tolist() == case["support"] and res["iters"] == case["iters"]
    assert np.allclose(res["x"], [_fr(v) for v in case["x"]], atol=1e-13)
    assert np.allclose(np.square(res["resnorm"]), [_fr(case["ynorm_sq"])] +
                       [_fr(t["rn_sq"]) for t in case["trace"] if t["accepted"]], atol=1e-13)


# ------------------------------------------- what each step defines
def _is_top(v, chosen, k, pool):
    """`chosen` is the k largest |v| over `pool` with ties to the lower index:
    every chosen j beats every pool member left out."""
    pool = [int(j) for j in pool]
    chosen = [int(j) for j in chosen]
    if len(chosen) != min(k, len(pool)) or not set(chosen) <= set(pool):
        return False
    a = np.abs(v) ** 2
    out = [j for j in pool if j not in chosen]
    return all(a[i] > a[o] or (a[i] == a[o] and i < o) for i in chosen for o in out)


def _ls_optimal(Phi, y, cols, x):
    """x solves the least squares on cols: the residual is orthogonal to them."""
    P = Phi[:, np.asarray(cols, dtype=np.int64)]
    return np.max(np.abs(P.conj().T @ (y - P @ x))) <= 1e-10 * np.linalg.norm(y)


def _noisy(kind, N, M, K, snr, seed):
    rng = np.random.default_rng(seed)
    om = synth.draw_omega(N, M, rng)
    Phi = matrices.sensing(kind, N, om)
    y = synth.add_noise(synth.measure(kind, N, om, synth.draw_support(N, K, rng),
                                      synth.draw_values(K, kind, "gauss", rng)), snr, rng)
    return Phi, y


# seeds 724 (WHT) and 735 (DFT) end on a rejected iterate whose support
# differs from the accepted one
SP_SEEDS = [700, 701, 702, 724, 735]
COSAMP_SEEDS = [800, 801, 802, 700, 811]  # 700 (WHT), 811 (DFT): the same for CoSaMP


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("seed", SP_SEEDS)
def test_sp_steps_follow_their_definitions(kind, seed):
    N, M, K = 128, 48, 6
    Phi, y = _noisy(kind, N, M, K, 12.0, seed)
    res = pursuits.subspace_pursuit(Phi, y, K)
    T, x, rn = res["T0"], res["x0"], res["resnorm"][0]
    assert _is_top(Phi.conj().T @ y, T, K, range(N)) and _ls_optimal(Phi, y, T, x)
    accepted = [rn]
    for st in res["trace"]:
        h = Phi.conj().T @ (y - Phi[:, T] @ x)
        new = sorted(set(st["Tp"].tolist()) - set(T.tolist()))
        assert set(T.tolist()) <= set(st["Tp"].tolist()) and len(st["Tp"]) == 2 * K
        assert _is_top(h, new, K, [j for j in range(N) if j not in set(T.tolist())])
        assert _ls_optimal(Phi, y, st["Tp"], st["b"])
        assert _is_top(st["b"], [i for i, j in enumerate(st["Tp"]) if j in set(st["Tn"].tolist())], K,
                       range(len(st["Tp"])))
        assert _ls_optimal(Phi, y, st["Tn"], st["x"])
        assert np.isclose(st["rn"], np.linalg.norm(y - Phi[:, st["Tn"]] @ st["x"]))
        assert st["accepted"] == (st["rn"] < rn)
        if not st["accepted"]:
            break
        T, x, rn = st["Tn"], st["x"], st["rn"]
        accepted.append(rn)
    assert res["support"].tolist() == T.tolist() and np.array_equal(res["x"], x)
    assert np.allclose(res["resnorm"], accepted)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("seed", COSAMP_SEEDS)
def test_cosamp_steps_follow_their_definitions(kind, seed):
    N, M, K = 128, 56, 5
    Phi, y = _noisy(kind, N, M, K, 12.0, seed)
    res = pursuits.cosamp(Phi, y, K)
    S, x, rn = np.zeros(0, np.int64), np.zeros(0, complex), np.linalg.norm(y)
    for st in res["trace"]:
        h = Phi.conj().T @ (y - (Phi[:, S] @ x if len(S) else 0))
        extra = sorted(set(st["T"].tolist()) - set(S.tolist()))
        top = pursuits.top_k(h, 2 * K)
        assert set(st["T"].tolist()) == set(top.tolist()) | set(S.tolist())
        assert _is_top(h, top, 2 * K, range(N)) and set(extra) <= set(top.tolist())
        assert _ls_optimal(Phi, y, st["T"], st["b"])
        keep = [i for i, j in enumerate(st["T"]) if j in set(st["S"].tolist())]
        assert _is_top(st["b"], keep, K, range(len(st["T"])))
        assert np.array_equal(st["x"], st["b"][keep])  # pruned, not solved again
        assert np.isclose(st["rn"], np.linalg.norm(y - Phi[:, st["S"]] @ st["x"]))
        assert st["accepted"] == (st["rn"] < rn)
        if not st["accepted"]:
            break
        S, x, rn = st["S"], st["x"], st["rn"]
    assert res["support"].tolist() == S.tolist() and np.array_equal(res["x"], x)
