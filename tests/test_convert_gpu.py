"""GPU parity: every conversion the library runs must equal the CPU oracle's
output byte for byte (pure data movement, no arithmetic), including the
padding, alignment holes and unused AoSoA slots, which the oracle defines as
zero.  Destinations start filled with garbage so that an unwritten byte
fails."""
import itertools

import numpy as np
import pytest

import datagen
import oracle
import paper_2511_04853_b300 as mrn
from gpu_util import (KINDS, dev, dev_dest, dev_view, garbage, host, oracle_pair, run,
                      torch)

pytestmark = pytest.mark.gpu

NESTED = [("a", "u8", 1),
          ("g", "group", [("x", "f64", 1), ("y", "u8", 1), ("h", "group", [("p", "u16", 3)])]),
          ("b", "u8", 1), ("c", "u32", 2)]
ODD = [("a", "u8", 1), ("b", "u16", 1)]                 # 4-byte record, 2-byte fields
TINY = [("a", "u8", 3)]                                 # 3-byte record: byte accesses
WIDE = [("v%d" % i, "f64" if i % 3 == 0 else "u16", 1) for i in range(40)]  # > 64-byte record
PACK2 = [("index", "u32", 1), ("weight", "f32", 1)]       # records of two 4-byte words
PACK4 = [("a", "i32", 1), ("v", "f32", 3)]                 # four 4-byte words (an array of 3)
PACK1 = [("x", "f32", 1)]                                  # one 4-byte word: tiles copied whole
PACK16 = [("t", "u16", 1), ("adc", "u16", 1)]              # one 4-byte word of two 2-byte columns
# Padding that no field can be stored wide enough to cover (byte b at 1 is
# not 2-aligned): AoS destination records keep their zeroing pass.  Points,
# sensor, nested and odd records instead absorb their padding in widened
# field stores.
UNCOV = [("a", "u8", 1), ("b", "u8", 1), ("c", "u32", 1)]


def schemas():
    return {"points": datagen.POINTS, "cells": datagen.CELLS, "sensor": datagen.SENSOR,
            "nested": NESTED, "odd": ODD, "tiny": TINY, "wide": WIDE, "pack2": PACK2, "pack4": PACK4,
            "pack1": PACK1, "pack16": PACK16, "uncov": UNCOV}


def data_for(name, n, seed=0, raw=False):
    if name in ("points", "cells"):
        return datagen.workload(name, n, seed, raw=raw)
    return datagen.random_columns(schemas()[name], n, seed)


def check_pair(name, n, sk, sb, dk, db, raw=False, seed=0):
    desc = schemas()[name]
    s, o = mrn.Schema(desc), oracle.Schema(desc)
    d = data_for(name, n, seed, raw)
    o_src, o_dst = oracle_pair(o, d, sk, sb, dk, db)
    src = dev_view(s, o_src, o)
    dst = dev_dest(s, dk, n, 0, db)
    run(src, dst)
    nbytes = o.base_bytes(dk, db, n)
    got = host(dst.tensors[0], nbytes)
    want = o_dst.base[:nbytes]
    if not np.array_equal(got, want):
        bad = np.nonzero(got != want)[0]
        raise AssertionError("%s n=%d %s(%d)->%s(%d): %d bytes differ, first at %d"
                             % (name, n, sk, sb, dk, db, bad.size, bad[0]))


PAIRS = [(a, b) for a, b in itertools.product(KINDS, KINDS) if a != b and not (a[0] == b[0] == "aos")]


@pytest.mark.parametrize("src,dst", PAIRS, ids=lambda k: "%s%d" % k)
@pytest.mark.parametrize("n", [0, 1, 31, 32, 33, 257, 1000])
def test_points_all_layout_pairs(src, dst, n):
    check_pair("points", n, src[0], src[1], dst[0], dst[1])


@pytest.mark.parametrize("name", ["cells", "sensor", "nested", "odd", "tiny", "wide", "uncov"])
@pytest.mark.parametrize("src,dst", [(("aos", 0), ("soa", 0)), (("soa", 0), ("aos", 0)),
                                     (("aos", 0), ("aosoa", 32)), (("aosoa", 32), ("aos", 0)),
                                     (("soa", 0), ("aosoa", 128)), (("aosoa", 128), ("aosoa", 32)),
                                     (("aosoa", 3), ("aos", 0)), (("aos", 0), ("aosoa", 5))],
                         ids=lambda k: "%s%d" % k)
@pytest.mark.parametrize("n", [1, 33, 4097])
def test_schemas_layout_pairs(name, src, dst, n):
    check_pair(name, n, src[0], src[1], dst[0], dst[1])


def test_points_10000_round_trip():
    """10,000 points: AoS -> SoA -> AoS reproduces the input bytes, and the SoA
    equals the oracle's (raw random bits too: NaN payloads, -0.0, denormals)."""
    for raw in (False, True):
        s, o = mrn.Schema(datagen.POINTS), oracle.Schema(datagen.POINTS)
        d = datagen.workload("points", 10000, 0, raw=raw)
        o_aos = oracle.pack(o, d, "aos")
        o_soa = oracle.convert(o, o_aos, "soa")
        src = dev_view(s, o_aos, o)
        soa = dev_dest(s, "soa", 10000)
        run(src, soa)
        assert np.array_equal(host(soa.tensors[0], o.base_bytes("soa", 0, 10000)), o_soa.base)
        back = dev_dest(s, "aos", 10000)
        run(soa, back)
        assert np.array_equal(host(back.tensors[0], 320000), o_aos.base)


@pytest.mark.parametrize("raw", [False, True])
def test_cells_200000_all_pairs(raw):
    """200,000 calorimeter cells: AoS <-> SoA <-> AoSoA(32), every direction."""
    n = 200000
    for (sk, sb), (dk, db) in [(("aos", 0), ("soa", 0)), (("soa", 0), ("aosoa", 32)),
                               (("aosoa", 32), ("aos", 0)), (("soa", 0), ("aos", 0)),
                               (("aos", 0), ("aosoa", 32)), (("aosoa", 32), ("soa", 0))]:
        check_pair("cells", n, sk, sb, dk, db, raw=raw, seed=1)


def test_per_column_pointer_views():
    """SoA given as separate column buffers (one allocation per property)."""
    n = 5000
    s, o = mrn.Schema(datagen.CELLS), oracle.Schema(datagen.CELLS)
    d = datagen.workload("cells", n, 1)
    o_aos = oracle.pack(o, d, "aos")
    cols = [garbage(n * c["size"]) for c in s.columns]
    src = dev_view(s, o_aos, o)
    dst = mrn.View(s, "soa", n, columns=cols)
    run(src, dst)
    want = oracle.flat_columns(d["columns"])
    for c in range(s.ncols):
        assert np.array_equal(host(cols[c]), want[c])
    back = dev_dest(s, "aos", n)
    run(mrn.View(s, "soa", n, columns=cols), back)
    assert np.array_equal(host(back.tensors[0], n * 24), o_aos.base)


def test_unaligned_aos_base_uses_narrow_accesses():
    """An AoS buffer starting 8 bytes past a 16-byte boundary."""
    n = 777
    s, o = mrn.Schema(datagen.POINTS), oracle.Schema(datagen.POINTS)
    d = datagen.workload("points", n, 3)
    o_aos = oracle.pack(o, d, "aos")
    o_soa = oracle.convert(o, o_aos, "soa")
    buf = dev(np.concatenate([np.zeros(8, np.uint8), o_aos.base]))
    src = mrn.View(s, "aos", n, base=buf.data_ptr() + 8)
    dst = dev_dest(s, "soa", n)
    run(src, dst)
    assert np.array_equal(host(dst.tensors[0], o.base_bytes("soa", 0, n)), o_soa.base)


def test_misaligned_column_rejected():
    s = mrn.Schema(datagen.CELLS)
    buf = garbage(24 * 10 + 16)
    src = mrn.View(s, "aos", 10, base=buf)
    cols = [buf.data_ptr() + 1] * s.ncols
    dst = mrn.View(s, "soa", 10, columns=cols)
    assert mrn.convert_status(src, dst) == mrn.EALIGN


@pytest.fixture
def direct_path():
    mrn.debug_set(3, 1)
    yield
    mrn.debug_set(3, 0)


@pytest.mark.parametrize("name", ["points", "cells", "sensor", "wide"])
@pytest.mark.parametrize("src,dst", [(("aos", 0), ("soa", 0)), (("soa", 0), ("aos", 0)),
                                     (("aos", 0), ("aosoa", 32)), (("aosoa", 128), ("soa", 0))],
                         ids=lambda k: "%s%d" % k)
def test_direct_path_parity(direct_path, name, src, dst):
    """The direct kernel (no TMA staging) gives the same bytes."""
    check_pair(name, 5000, src[0], src[1], dst[0], dst[1])


@pytest.mark.parametrize("n", [31, 32, 33, 383, 511, 512, 513, 543, 544, 545, 683, 1024 + 127, 1024 + 128,
                               1024 + 129, 2048, 100000])
def test_staged_tiles_and_tail(n):
    """Sizes around whole staged tiles (512 cell / 384 point records) and
    staging granules (32 records; 128 with AoSoA(128)): full tiles and the
    granule-aligned part of the last tile go through shared memory, the
    records after them through the direct path."""
    for (sk, sb), (dk, db) in [(("aos", 0), ("soa", 0)), (("soa", 0), ("aosoa", 128)),
                               (("aosoa", 32), ("aos", 0))]:
        check_pair("cells", n, sk, sb, dk, db, seed=7)
        check_pair("points", n, sk, sb, dk, db, seed=7)


@pytest.mark.parametrize("name,n", [("cells", 7_300_033), ("points", 5_500_017)])
def test_large_staged_conversions(name, n):
    """Conversions of at least 32 staged tiles per resident CTA (on a
    148-SM GPU: 7,274,496 cell or 5,455,872 point records) take guided
    chunks from a counter instead of a static split; a ragged size also
    ends in a partial tile."""
    for (sk, sb), (dk, db) in [(("aos", 0), ("soa", 0)), (("soa", 0), ("aosoa", 128)),
                               (("aosoa", 32), ("aos", 0))]:
        check_pair(name, n, sk, sb, dk, db, seed=11)


@pytest.mark.parametrize("name", ["pack1", "pack16", "pack2", "pack4"])
@pytest.mark.parametrize("n", [31, 32, 1000, 1536 * 3 + 64, 3072 * 2 + 96, 100003, 9_000_001])
def test_packed_records_aos_soa(name, n):
    """Records that are exactly one, two or four 4-byte words, or two
    2-byte columns, in column order, move between AoS and SoA as one word
    or vector per record in the staged transform (one 4-byte column: the
    tile copied whole); full tiles, partial tiles and the large-conversion
    path."""
    check_pair(name, n, "aos", 0, "soa", 0, seed=3)
    check_pair(name, n, "soa", 0, "aos", 0, seed=4)
    check_pair(name, n, "aos", 0, "aosoa", 32, seed=5)
