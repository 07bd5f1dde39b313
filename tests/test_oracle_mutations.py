"""Plants plausible slips in the oracle (on the CPU, through monkeypatch) and
checks that the pins of test_oracle_pins.py catch each one.  Nothing here
touches a GPU."""
import numpy as np
import pytest

import tests.test_oracle_pins as pins
from oracle import kernelsum, matrices, omp


def caught(fn, *a, **k):
    with pytest.raises(AssertionError):
        fn(*a, **k)


def test_wrong_dft_sign_is_caught(monkeypatch):
    def bad_fourier(N):
        i = np.arange(N)
        return np.exp(+2j * np.pi * (np.outer(i, i) % N) / N) / np.sqrt(N)
    monkeypatch.setattr(matrices, "fourier", bad_fourier)
    caught(pins.test_fourier_matches_fft, 8)


def test_missing_normalisation_is_caught(monkeypatch):
    orig = matrices.hadamard
    monkeypatch.setattr(matrices, "hadamard", lambda N: orig(N) * np.sqrt(N))
    caught(pins.test_unitary_and_unimodular, "wht", 8)


def test_dropped_conjugate_is_caught(monkeypatch):
    monkeypatch.setattr(omp, "correlate", lambda Phi, r: Phi.T @ r)
    caught(pins.test_correlation_is_adjoint, "dft")


def test_reversed_shift_is_caught(monkeypatch):
    def bad_shift(kind, N, j, lam):
        j = np.asarray(j, dtype=np.int64)
        return (lam - j) % N if kind == "dft" else j ^ lam
    monkeypatch.setattr(kernelsum, "shift_index", bad_shift)
    caught(pins.test_gram_is_shifted_kernel, "dft")
    caught(pins.test_fast_equals_conventional, "dft")


def test_transposed_kernel_definition_is_caught(monkeypatch):
    def bad_kernel(kind, N, omega):
        U = matrices.unitary(kind, N)
        S = matrices.row_selector(N, omega)
        e0 = np.zeros(N)
        e0[0] = 1
        return U @ (S.T @ (S @ (U.conj().T @ e0)))   # U and U^H swapped
    monkeypatch.setattr(kernelsum, "kernel_vector", bad_kernel)
    caught(pins.test_gram_is_shifted_kernel, "dft")


def test_highest_index_tie_break_is_caught(monkeypatch):
    def bad_identify(h, excluded):
        score = (np.conj(h) * h).real.astype(float).copy()
        if len(excluded):
            score[np.asarray(excluded)] = -np.inf
        j = len(score) - 1 - int(np.argmax(score[::-1]))
        return j, 1.0
    monkeypatch.setattr(omp, "identify", bad_identify)
    caught(pins.test_tiny_omp_by_hand)


def test_transposed_gram_in_least_squares_is_caught(monkeypatch):
    def bad_ls(Phi_t, y):
        G = Phi_t.T @ Phi_t          # missing conjugate
        b = Phi_t.conj().T @ y
        return np.linalg.solve(G, b), 1.0
    monkeypatch.setattr(omp, "least_squares", bad_ls)
    caught(pins.test_omp_invariants, "dft")


def test_dropped_kernel_term_is_caught(monkeypatch):
    orig = kernelsum.fast_correlation_dense
    bad_fast_impl = lambda kind, N, c, h0, support, x: orig(kind, N, c, h0, support[:-1], x[:-1])
    monkeypatch.setattr(kernelsum, "fast_correlation_dense", bad_fast_impl)
    caught(pins.test_fast_equals_conventional, "wht")


# --------------------------------------------- large-N (transform) oracle
def test_transform_forward_for_adjoint_is_caught(monkeypatch):
    import tests.test_oracle_transform as tpins
    from oracle import transform
    monkeypatch.setattr(transform, "apply_AH",
                        lambda kind, v: transform.apply_A(kind, v) if kind == "dft" else transform.fwht(v) / np.sqrt(v.shape[-1]))
    caught(tpins.test_correlate_and_synthesize_match_dense, "dft", 64, 20)


def test_transform_butterfly_slip_is_caught(monkeypatch):
    import tests.test_oracle_transform as tpins
    from oracle import transform

    def bad_fwht(v):
        a = np.array(v, dtype=float, copy=True)
        N = a.shape[-1]
        lead = a.shape[:-1]
        h = 1
        while h < N:
            a = a.reshape(*lead, N // (2 * h), 2, h)
            top, bot = a[..., 0, :], a[..., 1, :]
            a = np.stack((top + bot, bot - top), axis=-2)   # sign of the difference flipped
            h *= 2
        return a.reshape(*lead, N)
    monkeypatch.setattr(transform, "fwht", bad_fwht)
    caught(tpins.test_fwht_is_sylvester, 16)


def test_transform_residual_sign_is_caught(monkeypatch):
    import tests.test_oracle_transform as tpins
    from oracle import transform
    orig = transform.synthesize
    monkeypatch.setattr(transform, "synthesize", lambda *a: -orig(*a))
    caught(tpins.test_omp_matches_dense_oracle, "wht", 1024, 256, 16, None)


# ------------------------------------------------------ SP and CoSaMP
import inspect  # noqa: E402
import textwrap  # noqa: E402

import tests.test_oracle_pursuits as ppins  # noqa: E402
from oracle import pursuits  # noqa: E402


def _plant(monkeypatch, name, old, new):
    """Replace one statement of oracle.pursuits.<name> (the slip) and install
    the changed function in the module."""
    src = textwrap.dedent(inspect.getsource(getattr(pursuits, name)))
    assert src.count(old) == 1, old
    ns = dict(vars(pursuits))
    exec(compile(src.replace(old, new), f"<{name} with a slip>", "exec"), ns)
    monkeypatch.setattr(pursuits, name, ns[name])


def _sp_pins():
    for c in ppins.GOLD["sp"]:
        ppins.test_sp_iterates_by_hand(c)
    for kind in ppins.KINDS:
        for seed in ppins.SP_SEEDS:
            ppins.test_sp_steps_follow_their_definitions(kind, seed)


def _cosamp_pins():
    for c in ppins.GOLD["cosamp"]:
        ppins.test_cosamp_iterates_by_hand(c)
    for kind in ppins.KINDS:
        for seed in ppins.COSAMP_SEEDS:
            ppins.test_cosamp_steps_follow_their_definitions(kind, seed)


def test_pins_pass_on_the_oracle():
    _sp_pins()
    _cosamp_pins()


def test_sp_new_columns_over_all_j_is_caught(monkeypatch):
    _plant(monkeypatch, "subspace_pursuit", "top_k(h, K, excluded=T)", "top_k(h, K)")
    caught(_sp_pins)


def test_cosamp_second_least_squares_is_caught(monkeypatch):
    _plant(monkeypatch, "cosamp", "Sn, xn = T[keep], b[keep]", "Sn = T[keep]; xn = ls(Phi, y, Sn)")
    caught(_cosamp_pins)


def test_sp_accepting_an_equal_residual_is_caught(monkeypatch):
    _plant(monkeypatch, "subspace_pursuit", "if rn_new >= rn:", "if rn_new > rn:")
    caught(_sp_pins)


def test_cosamp_keeping_a_rejected_iterate_is_caught(monkeypatch):
    _plant(monkeypatch, "cosamp", "        if rn_new >= rn:\n            break\n        S, x, rn = Sn, xn, rn_new",
           "        rn_prev = rn\n        S, x, rn = Sn, xn, rn_new\n        if rn_new >= rn_prev:\n            break")
    caught(_cosamp_pins)


def test_sp_keeping_a_rejected_iterate_is_caught(monkeypatch):
    _plant(monkeypatch, "subspace_pursuit", "        if rn_new >= rn:\n            break\n        T, x, rn = Tn, xn, rn_new",
           "        rn_prev = rn\n        T, x, rn = Tn, xn, rn_new\n        if rn_new >= rn_prev:\n            break")
    caught(_sp_pins)
