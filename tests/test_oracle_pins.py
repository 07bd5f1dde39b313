"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each check is chosen so that a plausible slip in the oracle (a dropped
conjugate, a wrong DFT sign, a reversed shift, a missing 1/sqrt(N), a
transposed Gram matrix, a wrong tie-break) fails at least one of them; the
companion file test_oracle_mutations.py plants those slips and checks that
they are caught.
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import kernelsum, matrices, omp

GOLD = os.path.join(os.path.dirname(__file__), "golden")
KINDS = ["wht", "dft"]


def rand_vec(rng, n, kind):
    if kind == "dft":
        return rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return rng.standard_normal(n)


# ---------------------------------------------------------------- matrices --
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("N", [1, 2, 8, 64])
def test_unitary_and_unimodular(kind, N):
    """Sec. I constraint 1 (|U_ij| = 1/sqrt N) and unitarity."""
    U = matrices.unitary(kind, N)
    assert np.allclose(U.conj().T @ U, np.eye(N), atol=1e-12)
    assert np.allclose(np.abs(U), 1.0 / np.sqrt(N), atol=1e-14)


@pytest.mark.parametrize("kind", KINDS)
def test_columns_closed_under_product(kind):
    """Sec. I constraint 2: sqrt(N) u_a o sqrt(N) u_b is again some sqrt(N) u_c."""
    N = 16
    V = np.sqrt(N) * matrices.unitary(kind, N)
    for a in range(N):
        for b in range(N):
            p = V[:, a] * V[:, b]
            hits = [c for c in range(N) if np.allclose(p, V[:, c], atol=1e-12)]
            assert len(hits) == 1


def test_hadamard_kronecker_matches_closed_form():
    """The Kronecker-built Sylvester matrix equals (-1)^popcount(i&k)/sqrt(N),
    the closed form the instance generator evaluates."""
    N = 128
    H = matrices.hadamard(N)
    omega = np.arange(N, dtype=np.int32)
    for k in range(N):
        assert np.array_equal(H[:, k], synth.sensing_column("wht", N, omega, k))


@pytest.mark.parametrize("N", [2, 8, 256])
def test_fourier_matches_fft(N):
    """A x = fft(x)/sqrt(N): fixes the sign of the exponent and the scaling."""
    rng = np.random.default_rng(N)
    x = rand_vec(rng, N, "dft")
    assert np.allclose(matrices.fourier(N) @ x, np.fft.fft(x) / np.sqrt(N), atol=1e-12)


def test_sensing_is_row_subset():
    rng = np.random.default_rng(1)
    N, M = 64, 20
    om = synth.draw_omega(N, M, rng)
    for kind in KINDS:
        Phi = matrices.sensing(kind, N, om)
        assert np.array_equal(Phi, matrices.unitary(kind, N)[om])


# -------------------------------------------------------------- correlation --
@pytest.mark.parametrize("kind", KINDS)
def test_correlation_is_adjoint(kind):
    """<Phi^H r, v> = <r, Phi v>: pins the conjugate transpose of step 2)."""
    rng = np.random.default_rng(2)
    N, M = 64, 24
    om = synth.draw_omega(N, M, rng)
    Phi = matrices.sensing(kind, N, om)
    r = rand_vec(rng, M, "dft")
    v = rand_vec(rng, N, "dft")
    lhs = np.vdot(omp.correlate(Phi, r), v)
    rhs = np.vdot(r, Phi @ v)
    assert abs(lhs - rhs) < 1e-12 * (1 + abs(rhs))


@pytest.mark.parametrize("kind", KINDS)
def test_correlation_of_a_column(kind):
    """h = Phi^H phi_j has h(j) = ||phi_j||^2 = M/N, real and maximal."""
    rng = np.random.default_rng(3)
    N, M = 128, 40
    om = synth.draw_omega(N, M, rng)
    Phi = matrices.sensing(kind, N, om)
    for j in [0, 5, 77, N - 1]:
        h = omp.correlate(Phi, Phi[:, j])
        assert abs(h[j] - M / N) < 1e-13
        assert np.max(np.abs(h)) <= M / N + 1e-13


# ------------------------------------------------------------ kernel vector --
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("N,M", [(16, 5), (64, 16), (256, 100)])
def test_kernel_vector_identities(kind, N, M):
    """c(0) = M/N; sum |c|^2 = M/N (Parseval); DFT conjugate symmetry
    c(-d) = conj c(d) (Sec. III-B); WHT N c(d) integer with the parity of M
    (Sec. III-B: c takes few distinct values)."""
    rng = np.random.default_rng(N + M)
    om = synth.draw_omega(N, M, rng)
    c = kernelsum.kernel_vector(kind, N, om)
    assert abs(c[0] - M / N) < 1e-13
    assert abs(np.sum(np.abs(c) ** 2) - M / N) < 1e-12
    if kind == "dft":
        d = np.arange(N)
        assert np.allclose(c[(-d) % N], np.conj(c), atol=1e-13)
    else:
        nc = N * c
        assert np.allclose(nc, np.round(nc), atol=1e-10)
        assert np.all((np.round(nc).astype(int) - M) % 2 == 0)
        assert np.max(np.abs(nc)) <= M + 1e-9


@pytest.mark.parametrize("kind", KINDS)
def test_gram_is_shifted_kernel(kind):
    """(Phi^H Phi)(j, k) = c(j (-) k): the dense Gram equals the entries read
    off c.  Fixes the direction of the shift (j - k, not k - j)."""
    rng = np.random.default_rng(4)
    N, M = 64, 21
    om = synth.draw_omega(N, M, rng)
    Phi = matrices.sensing(kind, N, om)
    c = kernelsum.kernel_vector(kind, N, om)
    G = Phi.conj().T @ Phi
    all_idx = np.arange(N)
    assert np.allclose(G, kernelsum.gram_from_kernel(kind, N, c, all_idx), atol=1e-13)


@pytest.mark.parametrize("kind", KINDS)
def test_theorem_2_1_permutation(kind):
    """P_lambda = U^H D_lambda U is a 0/1 permutation matrix and sends c to
    the cyclic shift (Fourier) or XOR shift (Hadamard) of Sec. III-B."""
    N = 32
    for lam in [0, 1, 5, 17, N - 1]:
        P = kernelsum.permutation(kind, N, lam)
        Pr = np.round(P.real)
        assert np.allclose(P, Pr, atol=1e-12)
        assert np.all((Pr == 0) | (Pr == 1))
        assert np.all(Pr.sum(0) == 1) and np.all(Pr.sum(1) == 1)
        j = np.arange(N)
        cols = np.argmax(Pr, axis=1)
        assert np.array_equal(cols, kernelsum.shift_index(kind, N, j, lam))


@pytest.mark.parametrize("kind", KINDS)
def test_full_sampling_kernel_is_delta(kind):
    """Omega = [0, N): S^T S = I, so c = U^H U e_0 = e_0."""
    N = 32
    c = kernelsum.kernel_vector(kind, N, np.arange(N))
    e0 = np.zeros(N)
    e0[0] = 1
    assert np.allclose(c, e0, atol=1e-13)
    c_empty = kernelsum.kernel_vector(kind, N, np.zeros(0, dtype=np.int32))
    assert np.allclose(c_empty, 0)


def test_tiny_kernel_vectors_by_hand():
    g = json.load(open(os.path.join(GOLD, "tiny_by_hand.json")))
    for e in g["kernel_vectors"]:
        c = kernelsum.kernel_vector(e["kind"], e["N"], np.array(e["omega"]))
        want = np.array(e["c_re"]) + 1j * np.array(e["c_im"])
        assert np.allclose(c, want, atol=1e-14), e["derivation"]


# --------------------------------------------------------- fast correlation --
@pytest.mark.parametrize("kind", KINDS)
def test_fast_equals_conventional(kind):
    """Sec. III-A: h_0 - sum x(tau) P c equals Phi^H (y - Phi_Lambda x) for
    any support and coefficients (the method is exact)."""
    rng = np.random.default_rng(5)
    N, M, s = 64, 24, 7
    om = synth.draw_omega(N, M, rng)
    Phi = matrices.sensing(kind, N, om)
    y = rand_vec(rng, M, kind)
    lam = synth.draw_support(N, s, rng)
    x = rand_vec(rng, s, kind)
    c = kernelsum.kernel_vector(kind, N, om)
    h0 = kernelsum.initial_correlation(kind, N, om, y)
    assert np.allclose(h0, Phi.conj().T @ y, atol=1e-13)
    want = omp.correlate(Phi, y - Phi[:, lam] @ x)
    got_dense = kernelsum.fast_correlation_dense(kind, N, c, h0, lam, x)
    got_index = kernelsum.fast_correlation(kind, N, c, h0, lam, x)
    assert np.max(np.abs(got_dense - want)) < 1e-12
    assert np.max(np.abs(got_index - want)) < 1e-12


# ---------------------------------------------------------------------- OMP --
def test_tiny_omp_by_hand():
    g = json.load(open(os.path.join(GOLD, "tiny_by_hand.json")))
    for e in g["omp_runs"]:
        Phi = matrices.sensing(e["kind"], e["N"], np.array(e["omega"]))
        y = Phi @ np.array(e["x_true"])
        res = omp.omp(Phi, y, e["K"])
        assert res["support"] == e["support"], e["derivation"]
        assert np.allclose(res["x"], e["x"], atol=1e-12)
        assert res["iters"] == e["iters"]


@pytest.mark.parametrize("kind", KINDS)
def test_full_sampling_selects_in_magnitude_order(kind):
    """Omega = [0, N): Phi unitary, h_0 = x, so noiseless OMP picks the support
    in decreasing |x| and returns x exactly (closed form)."""
    rng = np.random.default_rng(6)
    N, K = 64, 6
    om = np.arange(N, dtype=np.int32)
    lam = synth.draw_support(N, K, rng)
    vals = synth.draw_values(K, kind, "gauss", rng)
    y = synth.measure(kind, N, om, lam, vals)
    res = omp.omp(matrices.sensing(kind, N, om), y, K)
    order = lam[np.argsort(-np.abs(vals), kind="stable")]
    assert res["support"] == order.tolist()
    xs = dict(zip(lam.tolist(), vals.tolist()))
    assert np.allclose(res["x"], [xs[j] for j in res["support"]], atol=1e-12)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_exact_noiseless_recovery(kind, seed):
    """K-sparse x from M >= 4 K log2(N/K) measurements is recovered exactly."""
    rng = np.random.default_rng(100 + seed)
    N, M, K = 256, 128, 8
    om = synth.draw_omega(N, M, rng)
    lam = synth.draw_support(N, K, rng)
    vals = synth.draw_values(K, kind, "gauss", rng)
    y = synth.measure(kind, N, om, lam, vals)
    res = omp.omp(matrices.sensing(kind, N, om), y, K)
    assert sorted(res["support"]) == sorted(lam.tolist())
    xs = dict(zip(lam.tolist(), vals.tolist()))
    assert np.allclose(res["x"], [xs[j] for j in res["support"]], atol=1e-10)
    assert res["resnorm"][-1] < 1e-10 * res["ynorm"]


@pytest.mark.parametrize("kind", KINDS)
def test_omp_invariants(kind):
    """After step 7) the residual is orthogonal to the chosen columns, so
    h_t(Lambda_t) = 0; ||r_t|| never grows; step 6) agrees with QR least squares."""
    rng = np.random.default_rng(7)
    N, M, K = 128, 48, 12
    om = synth.draw_omega(N, M, rng)
    Phi = matrices.sensing(kind, N, om)
    lam = synth.draw_support(N, K, rng)
    y = synth.add_noise(synth.measure(kind, N, om, lam, synth.draw_values(K, kind, "gauss", rng)), 20.0, rng)
    res = omp.omp(Phi, y, K, record_h=True)
    for t in range(1, res["iters"]):
        h = res["h"][t]
        assert np.max(np.abs(h[res["support"][:t]])) < 1e-12 * np.max(np.abs(res["h"][0]))
    rn = np.array(res["resnorm"])
    assert np.all(np.diff(rn) <= 1e-12 * rn[0])
    x_qr, *_ = np.linalg.lstsq(Phi[:, res["support"]], y, rcond=None)
    assert np.allclose(res["x"], x_qr, atol=1e-11)


def test_zero_measurement_halts_before_iterating():
    Phi = matrices.sensing("dft", 16, np.arange(8))
    res = omp.omp(Phi, np.zeros(8, complex), 4)
    assert res["iters"] == 0 and res["halt"] == "zero_y"


def test_dependent_column_stops():
    """Omega = {0, 2} of N = 4 (DFT): columns 0 and 2 coincide on those rows,
    so once one is chosen the other is dependent and the run stops."""
    Phi = matrices.sensing("dft", 4, np.array([0, 2]))
    # y = col 0 + col 1 : after two picks the residual is 0 (tolerance)
    y = Phi[:, 0] + 0.5 * Phi[:, 1]
    res = omp.omp(Phi, y, 4, rel_tol=0.0)
    assert res["iters"] == 2 and res["halt"] == "dependent"


@pytest.mark.parametrize("kind", KINDS)
def test_sensing_rows_match_dense(kind):
    rng = np.random.default_rng(8)
    N, M = 128, 50
    om = synth.draw_omega(N, M, rng)
    assert np.allclose(matrices.sensing_rows(kind, N, om), matrices.sensing(kind, N, om), atol=1e-13)
    assert np.allclose(kernelsum.kernel_vector_rows(kind, N, om), kernelsum.kernel_vector(kind, N, om), atol=1e-13)
