"""The C ABI library builds, loads without a GPU and exports every entry point of include/mlmc.h.

No compute call is made here (there may be no GPU); ctypes only resolves the symbols and
calls the one function that touches no device (the thread-local error string).
"""
import ctypes
import os
import re

import pytest

from paper_1904_00429_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mlmc.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^MLMC_API\s+[\w\s\*]+?\b(mlmc_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def so():
    build.build()
    return ctypes.CDLL(binding.LIB_PATH)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mlmc_plan", "mlmc_level_stats", "mlmc_estimate", "mlmc_backward"):
        assert required in names
    assert len(names) >= 15


def test_library_exports_every_declared_symbol(so):
    missing = [n for n in declared_functions() if not hasattr(so, n)]
    assert not missing, f"symbols declared in mlmc.h but not exported: {missing}"


def test_binding_signatures_cover_the_header():
    lib = binding.lib()
    for name in declared_functions():
        f = getattr(lib, name)
        assert f.restype is not None


def test_last_error_is_empty_before_any_call():
    assert binding.lib().mlmc_last_error() == b""


def test_struct_layouts_match_the_header():
    # int64 m,n,p; 2 ptr; int64; 2 ptr; int64; int32 x2; uint32 x4 -> 96 bytes on LP64
    assert ctypes.sizeof(binding.Problem) == 3 * 8 + 2 * 8 + 8 + 2 * 8 + 8 + 2 * 4 + 4 * 4
    assert ctypes.sizeof(binding.Options) == 4 * 4 + 8 + 8 + 8 + 4 + 4 + 4 + 4 + 4 + 4   # tail padding to 8
    assert ctypes.sizeof(binding.Report) == 8 + 32 * 8 * 4 + 3 * 8


def test_range_layout():
    # int32 prob, level; uint64 sample_begin, count
    assert ctypes.sizeof(binding.Range) == 24
