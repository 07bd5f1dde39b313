"""The C-ABI library loads and exports every symbol include/csfast.h
declares.  No compute call: runs without a GPU."""
import ctypes
import os
import re

import pytest

from paper_1205_4139_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "csfast.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cs_[a-z_0-9]+)\s*\(", txt)))


def test_header_and_binding_agree():
    assert declared_functions() == sorted(binding.EXPORTS)


@pytest.mark.skipif(not os.path.exists(binding.LIB_PATH), reason="library not built")
def test_library_exports_every_declared_symbol():
    L = ctypes.CDLL(binding.LIB_PATH)
    for name in declared_functions():
        assert hasattr(L, name), name


@pytest.mark.skipif(not os.path.exists(binding.LIB_PATH), reason="library not built")
def test_status_strings_without_gpu():
    L = binding.load()
    assert L.cs_status_string(0) == b"ok"
    assert L.cs_status_string(1) == b"invalid argument"


@pytest.mark.skipif(not os.path.exists(binding.LIB_PATH), reason="library not built")
def test_host_side_validation_without_gpu():
    """Argument checks run before any CUDA call, so they work on a CPU machine."""
    L = binding.load()
    h = ctypes.c_void_p()
    om = (ctypes.c_int32 * 3)(5, 3, 9)          # not sorted
    assert L.cs_plan_create(16, om, 3, 0, 0, None, ctypes.byref(h)) == 1
    om2 = (ctypes.c_int32 * 2)(1, 1)            # duplicate
    assert L.cs_plan_create(16, om2, 2, 0, 0, None, ctypes.byref(h)) == 1
    om3 = (ctypes.c_int32 * 1)(16)              # out of range
    assert L.cs_plan_create(16, om3, 1, 1, 1, None, ctypes.byref(h)) == 1
    assert L.cs_plan_create(12, om3, 1, 1, 1, None, ctypes.byref(h)) == 1   # N not a power of two
    assert L.cs_plan_create(16, om3, 17, 1, 1, None, ctypes.byref(h)) == 1  # M > N
    assert L.cs_plan_create(1 << 25, None, 0, 1, 1, None, ctypes.byref(h)) == 4  # beyond N limit (2^24)
    assert L.cs_plan_create(16, None, 0, 2, 1, None, ctypes.byref(h)) == 1   # bad kind
    assert L.cs_omp(None, None, 1, 4, None, None, None, None, None, None) == 1
    assert L.cs_omp_batched(None, -1, None, None, None, None, None, None, None, None) == 1  # negative count
    assert L.cs_omp_batched(None, 0, None, None, None, None, None, None, None, None) == 0   # empty batch
    assert L.cs_omp_batched(None, 2, None, None, None, None, None, None, None, None) == 1   # missing arrays
    bad = binding.Halt(-1.0, 2, -1, 0)
    assert L.cs_omp_batched(None, 0, None, None, ctypes.byref(bad), None, None, None, None, None) == 1
    one = (ctypes.c_void_p * 1)(None)
    k1 = (ctypes.c_int32 * 1)(1)
    assert L.cs_omp_batched(one, 1, one, k1, None, None, one, None, None, None) == 1  # NULL plan
    om4 = (ctypes.c_int32 * 2)(1, 5)
    assert L.cs_plan_create_ex(16, om4, 2, 0, 0, 1, None, ctypes.byref(h)) == 1   # half storage on a WHT plan
    assert L.cs_plan_create_ex(16, om4, 2, 1, 0, 2, None, ctypes.byref(h)) == 1   # integer storage on a DFT plan
    assert L.cs_plan_create_ex(16, om4, 2, 1, 0, 3, None, ctypes.byref(h)) == 1   # both
    assert L.cs_plan_create_ex(16, om4, 2, 1, 0, 8, None, ctypes.byref(h)) == 1   # unknown flag


def test_batch_wrapper_checks_arguments_on_the_host():
    """binding.Batch rejects mismatched lists and inputs that are not device
    vectors of the plan's length before it reaches the library."""
    torch = pytest.importorskip("torch")

    class FakePlan:
        M, kind, dtype = 8, "wht", torch.float64

    with pytest.raises(ValueError):
        binding.Batch([FakePlan()], [], [1])
    with pytest.raises(ValueError):  # a host tensor
        binding.Batch([FakePlan()], [torch.zeros(8, dtype=torch.float64)], [1])
