"""The paper-model flop counters reproduce the two numbers Sec. IV prints."""
import json
import os

from paper_1205_4139_gb300 import costmodel

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def test_excessive_point_fourier():
    e = GOLD["entries"][0]
    assert costmodel.excessive_point(e["kind"], e["N"]) == e["excessive_t"]
    t = e["conventional_from_t"]
    assert costmodel.fast_flops("dft", e["N"], t) > costmodel.conventional_flops("dft", e["N"])


def test_cosamp_ratio():
    e = GOLD["entries"][1]
    assert round(100 * costmodel.cosamp_fast_ratio(e["N"], e["K"])) == e["ratio_percent"]


def test_table_one_first_iteration_is_one_transform():
    for kind in ("dft", "wht"):
        assert costmodel.fast_flops(kind, 1024, 1) == costmodel.conventional_flops(kind, 1024)
    assert costmodel.conventional_flops("wht", 1024) == 2 * 1024 * 10
    assert costmodel.fast_flops("wht", 1024, 5) == 2 * 1024 * 4
    assert costmodel.fast_flops("dft", 4096, 3) == 6 * 4096 * 2


def test_omp_total():
    # all-fast vs all-conventional endpoints
    tot_conv = costmodel.omp_correlation_flops("dft", 4096, 64, 0)
    assert tot_conv == 64 * costmodel.conventional_flops("dft", 4096)
    tot_fast = costmodel.omp_correlation_flops("dft", 4096, 3, 99)
    assert tot_fast == costmodel.conventional_flops("dft", 4096) + 6 * 4096 * (1 + 2)
