"""The C-ABI library loads on a machine without a GPU and exports every entry
point include/ants.h declares; host-side argument checks work without one."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_1602_07247_gb300 as ants
from paper_1602_07247_gb300 import _build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ants.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"ANTS_API\s+[\w\s\*]+?\b(ants_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return C.CDLL(_build.LIB)


def test_header_declares_entry_points():
    syms = declared_symbols()
    for s in ("ants_ctx_create", "ants_lrf_create", "ants_lrf_load", "ants_reconstruct", "ants_last_error"):
        assert s in syms


def test_every_declared_symbol_is_exported(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_names_match_header():
    for s in declared_symbols():
        if s in ("ants_last_error", "ants_last_launch_count"):
            continue
        assert hasattr(ants, s), f"binding lacks {s}"


def test_version(lib):
    assert ants.ants_version() == 1


def test_detector_argument_checks(lib):
    with pytest.raises(ants.AntsError) as e:
        ants.ants_detector_create(np.zeros((0, 2)))
    assert e.value.code == -1 and "n_sensors" in str(e.value)
    with pytest.raises(ants.AntsError):
        ants.ants_detector_create(np.zeros((3, 2)), rel_gain=[1.0, 0.0, 1.0])
    with pytest.raises(ants.AntsError):
        ants.ants_detector_create(np.array([[0.0, np.nan]]))
    h = ants.ants_detector_create(np.zeros((3, 2)))
    ants.ants_detector_free(h)


def test_context_fails_loudly_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(ants.AntsError) as e:
        ants.ants_ctx_create(0)
    assert e.value.code == -2
