"""The C ABI library loads and exports every symbol include/*.h declares (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

import __graft_entry__  # noqa: F401  (puts the repo root on sys.path)
import paper_2204_06633_gb300 as lr
from paper_2204_06633_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        names += re.findall(r"LR_API\s+[\w\s\*]+?\b(lr_\w+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return lr.library()


def test_header_declares_the_expected_entry_points():
    names = declared_symbols()
    for must in ["lr_ctx_create", "lr_orbit_create", "lr_plan_create", "lr_project", "lr_tdi", "lr_response",
                 "lr_backward", "lr_response_batched", "lr_backward_batched", "lr_plan_check"]:
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
        assert name in lr._SIGS, f"binding has no signature for {name}"


def test_host_only_calls(lib):
    assert lr.strerror(0) == "success"
    assert "invalid" in lr.strerror(1)
    assert lib.lr_version() >= 100
    assert lr.order_supported(25)
    assert not lr.order_supported(24)
    assert not lr.order_supported(-1)


def test_null_arguments_are_rejected_on_the_host(lib):
    assert lib.lr_ctx_create(0, None) == 1
    assert lib.lr_plan_create(None, None, None) == 1
    assert lib.lr_orbit_destroy(None) == 1
    assert lib.lr_required_margin(None, None, None) == 1
    assert lib.lr_valid_range(None, None, None) == 1
    assert lib.lr_log_likelihood(None, None, None, 0, 0.0, lr.lr_sky(), None, None, None, None, None) == 1
    assert lib.lr_log_likelihood_batched(None, 1, None, None, None, None, None, None, None, 0, None, None, None,
                                         None) == 1
    assert lib.lr_likelihood(None, None, None, 0, 0.0, lr.lr_sky(), None, None, None, None, None) == 1
    assert lib.lr_likelihood_batched(None, 1, None, None, None, None, None, None, None, 0, None, None, None,
                                     None) == 1
