"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/bcgpu.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

from paper_1311_2147_gb300 import binding, build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "bcgpu.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bc_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_four_core_calls():
    names = declared_functions()
    for core in ("bc_init_static", "bc_apply_edge_update", "bc_apply_vertex_update", "bc_get_scores"):
        assert core in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    assert sorted(binding.EXPORTS) == declared_functions()


def test_binding_loads_and_sets_signatures():
    lib = binding.load()
    assert lib.bc_init_static.restype is ctypes.c_int


def test_record_layouts():
    assert binding.UPDATE_DTYPE.itemsize == 32
    assert binding.VEDGE_DTYPE.itemsize == 16
    assert ctypes.sizeof(binding.bc_info) == 176


def test_last_error_without_handle_is_empty_or_text():
    lib = binding.load()
    assert isinstance(lib.bc_last_error(None), bytes)


def test_encode_updates_layout():
    rec, ed = binding.encode_updates([("edge", 1, 2, 5), ("vertex", 3, [(4, 7, 0), (5, 8, 1)])])
    assert rec["kind"].tolist() == [0, 1] and rec["k"].tolist() == [0, 2] and rec["first"].tolist() == [0, 0]
    assert ed["x"].tolist() == [4, 5] and ed["dir"].tolist() == [0, 1] and ed["w"].tolist() == [7, 8]
