"""Host-side admission rule of the request runtime (cs_admit_next), no GPU:
oldest first, a later job may pass an oldest one that does not fit, and an
oldest job passed max_bypass times blocks everything behind it."""
import pytest

from paper_1205_4139_gb300 import binding


@pytest.fixture(scope="module", autouse=True)
def lib():
    try:
        binding.load()
    except RuntimeError as e:  # pragma: no cover
        pytest.skip(str(e))


def test_empty_queue():
    assert binding.admit_next([], [], 0, 100) == -1


def test_oldest_first_when_it_fits():
    assert binding.admit_next([30, 10, 10], [0, 0, 0], in_use=50, budget=100) == 0


def test_later_job_passes_an_oldest_that_does_not_fit():
    assert binding.admit_next([80, 60, 10], [0, 0, 0], in_use=50, budget=100) == 2


def test_nothing_fits():
    assert binding.admit_next([80, 60], [0, 0], in_use=50, budget=100) == -1


def test_no_pass_after_max_bypass():
    assert binding.admit_next([80, 10], [7, 0], in_use=50, budget=100, max_bypass=8) == 1
    assert binding.admit_next([80, 10], [8, 0], in_use=50, budget=100, max_bypass=8) == -1
    # ... but the oldest itself starts as soon as it fits
    assert binding.admit_next([80, 10], [8, 0], in_use=20, budget=100, max_bypass=8) == 0


def test_simulated_queue_never_starves_the_large_job():
    """Drive the rule the way the workers do: jobs finish in start order; a
    large job at the head must start within max_bypass admissions."""
    budget = 100
    pending = [90] + [20] * 40
    by = [0] * len(pending)
    running, started = [], []
    for _ in range(200):
        i = binding.admit_next(pending, by, sum(running), budget, 8)
        if i < 0:
            running.pop(0)  # the oldest running job finishes
            continue
        for k in range(i):
            by[k] += 1
        running.append(pending.pop(i))
        by.pop(i)
        started.append(running[-1])
        if not pending:
            break
    assert 90 in started[:9 + 1]
    assert not pending


def test_serving_request_stream_shape():
    import numpy as np
    import synth
    reqs = synth.serving_requests(400, rate=2000.0, seed=3)
    t = np.array([r["arrival_s"] for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert abs(np.mean(np.diff(t)) - 1 / 2000.0) < 0.2 / 2000.0  # Poisson at 2000/s
    for r in reqs:
        assert 1 << 14 <= r["N"] <= 1 << 20 and r["N"] & (r["N"] - 1) == 0
        assert r["M"] == r["N"] // 8 and 32 <= r["K"] <= 1024 and r["kind"] in ("wht", "dft")
    assert {r["N"] for r in reqs} == {1 << e for e in range(14, 21)}
    assert len({r["seed"] for r in reqs}) == len(reqs)
