"""Host-only checks of the C ABI: the library loads, exports every entry
point ``include/mrn.h`` declares, and its schema compiler and layout rules
agree with the oracle's (no GPU calls)."""
import ctypes
import os
import re

import numpy as np
import pytest

import datagen
import oracle
import paper_2511_04853_b300 as mrn
from paper_2511_04853_b300 import mrn as binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mrn.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mrn_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["mrn_schema_create", "mrn_schema_add_field", "mrn_schema_add_jagged",
                 "mrn_convert", "mrn_transfer_convert", "mrn_batch_create",
                 "mrn_autotune", "mrn_server_create", "mrn_server_submit", "mrn_sync"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    L = mrn.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    # and the binding declares a signature for each of them
    bound = {name for name, _, _ in binding.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_status_strings():
    assert mrn.status_str(mrn.OK) == "MRN_OK"
    assert mrn.status_str(mrn.EOVERFLOW) == "MRN_EOVERFLOW"


NESTED = [("a", "u8", 1),
          ("g", "group", [("x", "f64", 1), ("y", "u8", 1), ("h", "group", [("p", "u16", 3)])]),
          ("b", "u8", 1), ("c", "u32", 2)]
INTERLEAVED = [("id", "u32", 1), ("pos", "f32", 3, "interleaved"), ("flag", "u8", 1),
               ("g", "group", [("w", "u16", 4, "interleaved"), ("k", "u64", 2, "interleaved")]),
               ("c", "u8", 3, "interleaved"), ("plain", "u16", 2)]
INTERLEAVED_JAGGED = [("pt", "f32", 1), ("cov", "f32", 3, "interleaved"),
                      ("hits", "jagged", "u32", [("index", "u32", 1), ("weight", "f32", 1)])]
ALL = {"points": datagen.POINTS, "cells": datagen.CELLS, "tracks": datagen.TRACKS,
       "sensor": datagen.SENSOR, "particle": datagen.PARTICLE, "nested": NESTED,
       "interleaved": INTERLEAVED, "interleaved_jagged": INTERLEAVED_JAGGED}


@pytest.mark.parametrize("name", sorted(ALL))
def test_schema_compiler_matches_oracle(name):
    desc = ALL[name]
    s, o = mrn.Schema(desc), oracle.Schema(desc)
    assert s.stride == o.stride
    assert [c["aos_offset"] for c in s.columns] == o.col_aos_off
    assert [c["size"] for c in s.columns] == o.col_size
    assert [c["fm_stride"] for c in s.columns] == o.col_es
    assert s.has_jagged == o.has_jagged
    if s.has_jagged:
        assert s.info.jag_length_offset == o.len_off
        assert s.info.jag_begin_offset == o.begin_off
        assert s.info.offset_size == o.off_size
        assert s.info.child_stride == o.child.stride
        assert [c["aos_offset"] for c in s.child_columns] == o.child.col_aos_off
    for n, m in [(0, 0), (1, 0), (10000, 5), (200001, 77)]:
        assert s.required_bytes("aos", n, m) == o.base_bytes("aos", 0, n, m)
        assert s.required_bytes("soa", n, m) == o.base_bytes("soa", 0, n, m)
        nreg = s.ncols + (1 + len(s.child_columns) if s.has_jagged else 0)
        for r in range(nreg):
            assert s.soa_region_offset(n, m, r) == o.soa_region_start(n, m, r)
        for B in (1, 3, 32, 128):
            assert s.required_bytes("aosoa", n, m, B) == o.base_bytes("aosoa", B, n, m)
            assert s.aosoa_block_bytes(B) == o.aosoa_block_bytes(B)
            for c in range(s.ncols):
                assert s.aosoa_column_offset(B, c) == o.aosoa_col_start(B, c)


def test_interleaved_child_schema_is_refused():
    child = mrn.Schema([("x", "f32", 3, "interleaved")])
    L = mrn.lib()
    h = ctypes.c_void_p()
    assert L.mrn_schema_create(ctypes.byref(h)) == 0
    assert L.mrn_schema_add_jagged(h, b"v", 4, child._h) == mrn.EUNSUPPORTED
    L.mrn_schema_destroy(h)


def test_interleaved_hash_differs_from_separate_columns():
    a = mrn.Schema([("v", "u16", 4)])
    b = mrn.Schema([("v", "u16", 4, "interleaved")])
    assert a.hash != b.hash and a.stride == b.stride


def test_column_names_follow_the_description():
    s = mrn.Schema(datagen.PARTICLE)
    names = [c["name"] for c in s.columns]
    assert names[:4] == ["energy", "x", "y", "origin"]
    assert "significance[3]" in names and "noisy_count[0]" in names
    s2 = mrn.Schema(datagen.SENSOR)
    assert "calibration_data.noise_B" in [c["name"] for c in s2.columns]


@pytest.mark.parametrize("bad", [
    [],
    [("x", "u8", 0)],
    [("v", "jagged", "u16", [("x", "u8", 1)])],
    [("v", "jagged", "u32", [("x", "u8", 1)]), ("w", "jagged", "u32", [("x", "u8", 1)])],
    [("v", "jagged", "u32", [("c", "jagged", "u32", [("d", "jagged", "u32", [("x", "u8", 1)])])])],
])
def test_invalid_schemas_are_rejected(bad):
    with pytest.raises(mrn.MrnError) as e:
        mrn.Schema(bad)
    assert e.value.code == mrn.EINVAL


def test_unclosed_group_rejected():
    L = mrn.lib()
    h = ctypes.c_void_p()
    assert L.mrn_schema_create(ctypes.byref(h)) == 0
    assert L.mrn_schema_begin_group(h, b"g") == 0
    assert L.mrn_schema_add_field(h, b"x", 4, 1) == 0
    assert L.mrn_schema_finalize(h) == mrn.EINVAL
    assert L.mrn_schema_end_group(h) == 0
    assert L.mrn_schema_finalize(h) == 0
    assert L.mrn_schema_add_field(h, b"y", 4, 1) == mrn.EINVAL  # immutable
    L.mrn_schema_destroy(h)


def test_hash_is_structural():
    a = mrn.Schema(datagen.CELLS)
    b = mrn.Schema([(n + "_renamed", t, e) for n, t, e in datagen.CELLS])
    c = mrn.Schema(datagen.POINTS)
    assert a.hash == b.hash and a.hash != c.hash


def test_convert_rejects_bad_views_without_a_device():
    s = mrn.Schema(datagen.CELLS)
    buf = np.zeros(24 * 10, np.uint8)
    src = mrn.View(s, "aos", 10, base=buf, mem="host")
    dst = mrn.View(s, "soa", 11, base=buf, mem="host")
    # n mismatch is rejected on the host before anything touches a device
    assert mrn.convert_status(src, dst, stream=0) == mrn.EINVAL
    dst2 = mrn.View(s, "aosoa", 10, block=0, base=buf, mem="host")
    assert mrn.convert_status(src, dst2, stream=0) == mrn.EINVAL


def test_scratch_release_without_a_device():
    """No pool exists before a conversion: the release is a no-op; a device
    index outside 0..63 is refused."""
    mrn.scratch_release(0)
    with pytest.raises(mrn.MrnError) as e:
        mrn.scratch_release(64)
    assert e.value.code == mrn.EINVAL


@pytest.mark.parametrize("desc", [datagen.TRACKS_NESTED,
                                  [("g", "group", [("p", "f64", 1),
                                                   ("v", "jagged", "u32", [("x", "u8", 2),
                                                                           ("w", "jagged", "u64",
                                                                            [("y", "u16", 1)])])])]])
def test_nested_layout_matches_oracle(desc):
    s, o = mrn.Schema(desc), oracle.Schema(desc)
    assert s.stride == o.stride and s.info.child_stride == o.child.stride
    items = s.ncols + 1 + len(s.child_columns) + 1 + len(o.child.child.col_size)
    for n, m, m2 in [(0, 0, 0), (1, 3, 7), (1000, 20011, 60001)]:
        for kind, B in (("soa", 0), ("aosoa", 1), ("aosoa", 32)):
            assert s.required_bytes_nested(kind, n, m, m2, B) == o.base_bytes(kind, B, n, m, m2)
            nit = items if kind == "soa" else 2 + len(s.child_columns) + 1 + len(o.child.child.col_size)
            for r in range(nit):
                assert s.region_offset_nested(kind, n, m, m2, r, B) == o.fm_region_start(kind, B, n, m, r, m2), \
                    (kind, B, n, m, m2, r)
        assert s.grandchild_pool_bytes(m2) == m2 * o.child.child.stride


def test_nesting_deeper_than_once_is_refused():
    inner = mrn.Schema([("x", "u8", 1), ("w", "jagged", "u32", [("y", "u8", 1)])])
    mid = mrn.Schema([("z", "u8", 1), ("v", "jagged", "u32", [("x", "u8", 1), ("w", "jagged", "u32",
                                                                                 [("y", "u8", 1)])])])
    L = mrn.lib()
    h = ctypes.c_void_p()
    assert L.mrn_schema_create(ctypes.byref(h)) == 0
    assert L.mrn_schema_add_jagged(h, b"ok", 4, inner._h) == 0
    L.mrn_schema_destroy(h)
    assert L.mrn_schema_create(ctypes.byref(h)) == 0
    assert L.mrn_schema_add_jagged(h, b"deep", 4, mid._h) == mrn.EINVAL
    L.mrn_schema_destroy(h)
