"""Host-side fault injection and failing loudly without a GPU (no GPU needed).

MLMC_FAULT=alloc makes mlmc_plan fail as a device allocation would, before any CUDA call, so
the error path (status code, message, no exception across the ABI) is checked on the CPU.
Without the injection, mlmc_plan on a machine without a usable GPU reports MLMC_ERR_CUDA: the
library never falls back to the CPU.
"""
import ctypes

import pytest
import torch

from paper_1904_00429_gb300 import binding, build


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def _problem():
    # sizes and non-null pointers pass validation; they are never dereferenced on these paths
    dummy = 0x1000
    return binding.Problem(8, 16, 8, dummy, dummy, 16, dummy, dummy, 8, 1, -1, 0, 1, 2, 0)


def _plan_status():
    arr = (binding.Problem * 1)(_problem())
    opts = binding.Options(4, 2, 2, binding.PRECISION["fp32"], 8, 1.0, 0, 0, 0)
    h = ctypes.c_void_p()
    st = binding.lib().mlmc_plan(arr, 1, ctypes.byref(opts), None, ctypes.byref(h))
    return st, h, binding.lib().mlmc_last_error().decode()


def test_injected_allocation_failure(monkeypatch):
    monkeypatch.setenv("MLMC_FAULT", "alloc")
    st, h, msg = _plan_status()
    assert st == 3 and h.value is None
    assert "injected" in msg


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the behaviour without a GPU")
def test_plan_fails_loudly_without_a_gpu(monkeypatch):
    monkeypatch.delenv("MLMC_FAULT", raising=False)
    st, h, msg = _plan_status()
    assert st == 2 and h.value is None
    assert msg


def test_invalid_arguments_are_reported_before_anything_else(monkeypatch):
    monkeypatch.setenv("MLMC_FAULT", "alloc")
    arr = (binding.Problem * 1)(_problem())
    opts = binding.Options(0, 2, 2, binding.PRECISION["fp32"], 8, 1.0, 0, 0, 0)   # c0 = 0
    h = ctypes.c_void_p()
    st = binding.lib().mlmc_plan(arr, 1, ctypes.byref(opts), None, ctypes.byref(h))
    assert st == 1
    assert "c0" in binding.lib().mlmc_last_error().decode()


@pytest.mark.parametrize("fields,status,word", [
    # (precision, f, adaptive_L, sampling) -> status, a word of the message
    (("fp32", 7, 0, 0), 1, "unknown f"),  # unknown targeted function
    (("fp32", 0, 2, 0), 1, "adaptive_L"),
    (("fp32", 0, 0, 5), 1, "sampling"),
    (("fp8", 1, 0, 0), 6, "FP64, FP32 or BF16"),   # f has no E4M3 form
    (("fp8", 0, 0, 1), 6, "FP64, FP32 or BF16"),   # xi** has no E4M3 form
])
def test_option_combinations_are_validated_on_the_host(monkeypatch, fields, status, word):
    """Targeted function, adaptive L and sampling law are checked before any device work (the
    injected allocation fault would otherwise be reported)."""
    monkeypatch.setenv("MLMC_FAULT", "alloc")
    prec, f, adaptive, sampling = fields
    arr = (binding.Problem * 1)(_problem())
    opts = binding.Options(4, 2, 2, binding.PRECISION[prec], 8, 1.0, 0, 0, 0, f, adaptive, sampling)
    h = ctypes.c_void_p()
    st = binding.lib().mlmc_plan(arr, 1, ctypes.byref(opts), None, ctypes.byref(h))
    assert st == status and h.value is None
    assert word in binding.lib().mlmc_last_error().decode()


def test_valid_new_options_pass_validation(monkeypatch):
    monkeypatch.setenv("MLMC_FAULT", "alloc")
    for prec in ("fp64", "fp32"):
        arr = (binding.Problem * 1)(_problem())
        opts = binding.Options(4, 2, 2, binding.PRECISION[prec], 8, 1.0, 0, 0, 0, 1, 1, 1)
        h = ctypes.c_void_p()
        st = binding.lib().mlmc_plan(arr, 1, ctypes.byref(opts), None, ctypes.byref(h))
        assert st == 3   # reached the (injected) allocation: validation accepted f, adaptive L and xi**


def test_generation_rate_rejects_a_null_output():
    st = binding.lib().mlmc_measure_generation_rate(None, None)
    assert st == 1
