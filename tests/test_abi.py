"""CPU checks of the C ABI: the library loads, exports what include/vdmc.h
declares, and its host-side class tables agree with the oracle's.

No device call is made here.  The library builds its class table by orbit
closure under adjacent transpositions; the oracle by trying all k!
permutations -- two independent constructions of the same table.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT
from oracle import oracle as O
from paper_2201_11655_b300 import build, vdmc


def declared_functions():
    text = open(os.path.join(ROOT, "include", "vdmc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vdmc_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return vdmc.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    raw = ctypes.CDLL(vdmc.LIB_PATH)
    for name in names:
        assert hasattr(raw, name), name


def test_num_classes(lib):
    assert vdmc.num_classes(3) == 13
    assert vdmc.num_classes(4) == 199
    assert vdmc.num_classes(2) == -1
    assert vdmc.num_classes(5) == -1


@pytest.mark.parametrize("k", [3, 4])
def test_class_tables_match_oracle(lib, k):
    canon, _ = O.classes(k)
    np.testing.assert_array_equal(vdmc.class_masks(k).astype(np.int64), canon)
    lut = vdmc.class_lut(k)
    for idx in range(1 << (k * (k - 1))):
        c = O.canonical_index(k, idx)
        hit = np.nonzero(canon == c)[0]
        want = int(hit[0]) if hit.size else 255
        assert lut[idx] == want, idx


def test_status_strings(lib):
    for s in range(7):
        assert lib.vdmc_status_string(s)
    assert lib.vdmc_status_string(99) == b"unknown status"


def test_invalid_args_rejected_on_host(lib):
    h = ctypes.c_void_p()
    # negative n, n >= 2^30, NULL arc pointers with m > 0 -- all refused before
    # any device work
    assert lib.vdmc_graph_create(-1, 0, None, None, 0, None, ctypes.byref(h)) == 1
    assert lib.vdmc_graph_create(1 << 30, 0, None, None, 0, None, ctypes.byref(h)) == 1
    assert lib.vdmc_graph_create(5, 3, None, None, 0, None, ctypes.byref(h)) == 1
    assert lib.vdmc_count(None, 3, None, None) == 1
    assert lib.vdmc_graph_info(None, None) == 1
    s = vdmc.Schedule(0, 8, 0, 0, 1)
    assert lib.vdmc_set_schedule(ctypes.byref(s)) == 1
    s = vdmc.Schedule(4, 8, 0, 0, 0)  # hub_blocks_per_sm must be >= 1
    assert lib.vdmc_set_schedule(ctypes.byref(s)) == 1


def test_schedule_roundtrip(lib):
    old = vdmc.get_schedule()
    try:
        vdmc.set_schedule(a_chunk=3, warps_per_block=4, blocks_per_sm=2, hub_min_l=7, hub_blocks_per_sm=2,
                          hub_split=4, hub_split_roots=9, hub_warps=32, d3_bits=64)
        assert vdmc.get_schedule() == {"a_chunk": 3, "warps_per_block": 4, "blocks_per_sm": 2,
                                       "hub_min_l": 7, "hub_blocks_per_sm": 2, "hub_split": 4, "hub_split_roots": 9,
                                       "hub_warps": 32, "d3_bits": 64}
        for bad in ({"hub_split": -1}, {"hub_split": 17}, {"hub_split_roots": -1}, {"hub_warps": 8},
                    {"d3_bits": 32}):
            with pytest.raises(vdmc.VdmcError):
                vdmc.set_schedule(**bad)
    finally:
        vdmc.set_schedule(**old)


@pytest.mark.parametrize("k", [3, 4])
def test_undirected_class_tables_match_oracle(lib, k):
    # the library keeps the directed classes of symmetric matrices; the
    # oracle enumerates symmetric connected matrices directly
    canon, _ = O.classes_undirected(k)
    assert vdmc.num_classes_undirected(k) == len(canon)
    np.testing.assert_array_equal(vdmc.undirected_class_masks(k).astype(np.int64), canon)
    assert vdmc.num_classes_undirected(5) == -1
