"""Pins the CPU oracle to things other than itself.

* numpy's aligned structured dtypes (the C compiler's layout rules) for the
  AoS record and the AoSoA block, and numpy field access for the columns;
* round-trip identities between layouts;
* closed forms: all-equal field sizes make AoS->SoA a matrix transpose, a
  single-field schema makes every layout a plain copy;
* the jagged offsets invariants and numpy's cumsum / concatenation for the
  flattened child values (Sec. V, jagged vector property);
* brute force over every small schema, with unique byte values, so that a
  lost, duplicated or misplaced byte fails.
"""
import itertools

import numpy as np
import pytest

import datagen
import oracle
from np_layout import (struct_dtype, aos_from_values, aos_columns,
                       block_dtype, aosoa_columns, fill_block_column)

# a sub-group that needs alignment and tail padding of its own
NESTED = [("a", "u8", 1),
          ("g", "group", [("x", "f64", 1), ("y", "u8", 1),
                          ("h", "group", [("p", "u16", 3)])]),
          ("b", "u8", 1), ("c", "u32", 2)]

SCHEMAS = {"points": datagen.POINTS, "cells": datagen.CELLS,
           "sensor": datagen.SENSOR, "nested": NESTED}


def values_for(desc, n, seed):
    return datagen.random_columns(desc, n, seed)


# ---------------------------------------------------------------- AoS rules

@pytest.mark.parametrize("name", ["points", "cells", "sensor", "nested", "tracks", "particle"])
def test_aos_offsets_match_numpy_aligned_struct(name):
    desc = {"points": datagen.POINTS, "cells": datagen.CELLS,
            "sensor": datagen.SENSOR, "nested": NESTED, "tracks": datagen.TRACKS,
            "particle": datagen.PARTICLE}[name]
    s = oracle.Schema(desc)
    dt = struct_dtype(desc)
    assert s.stride == dt.itemsize
    # numpy offsets of the flattened leaves
    offs = []

    def walk(d, base):
        for fname in d.names:
            sub, off = d.fields[fname][0], d.fields[fname][1]
            if sub.names is not None:
                walk(sub, base + off)
            elif fname.endswith("_length") or fname.endswith("_begin"):
                continue
            elif sub.shape:
                offs.extend(base + off + k * sub.base.itemsize for k in range(sub.shape[0]))
            else:
                offs.append(base + off)
    walk(dt, 0)
    assert s.col_aos_off == offs
    if s.has_jagged:
        jn = datagen.jagged_member(desc)[0]
        assert s.len_off == dt.fields[jn + "_length"][1]
        assert s.begin_off == dt.fields[jn + "_begin"][1]


def test_workload_strides():
    # the three workload records: 32-byte points with 7 bytes of padding,
    # 24-byte cells, 24-byte tracks with the {length, begin} descriptor
    assert oracle.Schema(datagen.POINTS).stride == 32
    assert oracle.Schema(datagen.POINTS).col_aos_off == [0, 4, 8, 12, 16, 24]
    assert oracle.Schema(datagen.CELLS).stride == 24
    t = oracle.Schema(datagen.TRACKS)
    assert (t.stride, t.len_off, t.begin_off, t.child.stride) == (24, 12, 16, 8)


@pytest.mark.parametrize("name", list(SCHEMAS))
@pytest.mark.parametrize("n", [0, 1, 5, 33, 1000])
def test_soa_to_aos_equals_numpy_fill(name, n):
    desc = SCHEMAS[name]
    s = oracle.Schema(desc)
    d = values_for(desc, n, 11)
    aos = oracle.pack(s, d, "aos")
    ref = aos_from_values(desc, d["columns"], n)
    assert aos.base[: n * s.stride].tobytes() == ref.tobytes()


@pytest.mark.parametrize("name", list(SCHEMAS))
@pytest.mark.parametrize("n", [0, 1, 7, 129, 1000])
def test_aos_to_soa_equals_numpy_fields(name, n):
    desc = SCHEMAS[name]
    s = oracle.Schema(desc)
    ref = aos_from_values(desc, values_for(desc, n, 3)["columns"], n)
    raw = np.frombuffer(ref.tobytes(), np.uint8).copy() if n else np.zeros(1, np.uint8)
    soa = oracle.convert(s, oracle.Side("aos", n, base=raw), "soa")
    cols = aos_columns(desc, raw, n)
    for c in range(s.ncols):
        assert oracle.region(s, soa, c).tobytes() == cols[c].tobytes()
    # every byte of the block outside the columns is zero
    mask = np.ones(soa.base.size, bool)
    for c in range(s.ncols):
        st = s.soa_region_start(n, 0, c)
        mask[st:st + n * s.col_size[c]] = False
        assert st % 128 == 0
    assert not soa.base[mask].any()


# ------------------------------------------------------------- AoSoA rules

@pytest.mark.parametrize("name", list(SCHEMAS))
@pytest.mark.parametrize("B", [1, 3, 8, 32, 128])
@pytest.mark.parametrize("n", [0, 1, 31, 32, 33, 300])
def test_aosoa_matches_numpy_block_struct(name, B, n):
    desc = SCHEMAS[name]
    s = oracle.Schema(desc)
    d = values_for(desc, n, 5)
    assert s.aosoa_block_bytes(B) == block_dtype(desc, B).itemsize
    out = oracle.pack(s, d, "aosoa", B)
    cols, blocks = aosoa_columns(desc, out.base, n, B)
    want = oracle.flat_columns(d["columns"])
    for c in range(s.ncols):
        assert cols[c].view(np.uint8).tobytes() == want[c].tobytes()
    # tail slots of the last block and every alignment hole are zero:
    # rebuild the blocks from the columns with numpy and compare all bytes
    ref = np.zeros(len(blocks), block_dtype(desc, B))
    for c in range(s.ncols):
        fill_block_column(ref, c, cols[c], n)
    assert out.base[: ref.nbytes].tobytes() == ref.tobytes()


# ------------------------------------------------------------ round trips

@pytest.mark.parametrize("name", list(SCHEMAS))
@pytest.mark.parametrize("n", [0, 1, 100, 4097])
def test_round_trips_identity(name, n):
    desc = SCHEMAS[name]
    s = oracle.Schema(desc)
    d = values_for(desc, n, 21)
    aos = oracle.pack(s, d, "aos")
    a = oracle.convert(s, oracle.convert(s, aos, "soa"), "aos")
    assert a.base.tobytes() == aos.base.tobytes()
    b = oracle.convert(s, oracle.convert(s, oracle.convert(s, aos, "aosoa", 32), "soa"), "aos")
    assert b.base.tobytes() == aos.base.tobytes()
    soa = oracle.convert(s, aos, "soa")
    c = oracle.convert(s, oracle.convert(s, oracle.convert(s, soa, "aosoa", 32), "aosoa", 128), "soa")
    assert c.base.tobytes() == soa.base.tobytes()
    via = oracle.convert(s, oracle.convert(s, aos, "aosoa", 8), "soa")
    assert via.base.tobytes() == soa.base.tobytes()


# ------------------------------------------------------------ closed forms

@pytest.mark.parametrize("size,dt", [(1, "u8"), (2, "u16"), (4, "f32"), (8, "u64")])
@pytest.mark.parametrize("F", [1, 3, 5])
def test_equal_sizes_is_a_transpose(size, dt, F):
    desc = [("f%d" % k, dt, 1) for k in range(F)]
    s = oracle.Schema(desc)
    n = 77
    d = values_for(desc, n, 9)
    aos = oracle.pack(s, d, "aos")
    mat = aos.base.view(np.dtype("<u%d" % size)).reshape(n, F)
    soa = oracle.convert(s, aos, "soa")
    for c in range(F):
        assert oracle.region(s, soa, c).view(mat.dtype).tolist() == mat.T[c].tolist()


@pytest.mark.parametrize("dt", ["u8", "u16", "f32", "f64"])
def test_single_field_every_layout_is_a_copy(dt):
    desc = [("v", dt, 1)]
    s = oracle.Schema(desc)
    n = 64
    d = values_for(desc, n, 4)
    raw = d["columns"][0].view(np.uint8).tobytes()
    for kind, B in [("aos", 0), ("soa", 0), ("aosoa", 16), ("aosoa", 64)]:
        out = oracle.pack(s, d, kind, B)
        assert out.base.tobytes()[: len(raw)] == raw


def test_array_property_is_extent_columns():
    # an array property of extent E is E per-index columns (Sec. V)
    desc = [("a", "u16", 3), ("b", "u8", 1)]
    s = oracle.Schema(desc)
    assert s.ncols == 4 and s.col_size == [2, 2, 2, 1]
    n = 10
    d = values_for(desc, n, 8)
    soa = oracle.convert(s, oracle.pack(s, d, "aos"), "soa")
    for k in range(3):
        assert oracle.region(s, soa, k).view("<u2").tolist() == d["columns"][0][:, k].tolist()


# ------------------------------------------------------------------ jagged

def _tracks(n, seed, **kw):
    s = oracle.Schema(datagen.TRACKS)
    return s, datagen.workload("tracks", n, seed, **kw)


@pytest.mark.parametrize("n", [0, 1, 5, 1000])
def test_offsets_invariants_and_children(n):
    s, d = _tracks(n, 2)
    order = np.random.default_rng(7).permutation(n)
    aos = oracle.shuffle_pool(s, oracle.pack(s, d, "aos"), order, gap=1)
    soa = oracle.convert(s, aos, "soa", m=d["m"])
    off = oracle.region(s, soa, s.ncols).view(np.uint32).astype(np.int64)
    lens = d["lengths"].astype(np.int64)
    assert off[0] == 0 and (np.diff(off) >= 0).all()
    assert off[-1] == lens.sum() == d["m"] == soa.written
    assert off.tolist() == np.concatenate([[0], np.cumsum(lens)]).tolist()
    # children: concatenation of every parent's slice of the shuffled pool
    pool = np.frombuffer(aos.pool[: aos.m * 8].tobytes(), struct_dtype([("index", "u32", 1), ("weight", "f32", 1)]))
    recs = np.frombuffer(aos.base[: n * 24].tobytes(), struct_dtype(datagen.TRACKS), count=n)
    parts = [pool[int(b):int(b) + int(L)] for b, L in zip(recs["hits_begin"], recs["hits_length"])]
    kids = np.concatenate(parts) if parts else pool[:0]
    assert oracle.region(s, soa, s.ncols + 1).tobytes() == np.ascontiguousarray(kids["index"]).tobytes()
    assert oracle.region(s, soa, s.ncols + 2).tobytes() == np.ascontiguousarray(kids["weight"]).tobytes()
    # parent columns through numpy field access
    for c, name in enumerate(["pt", "eta", "label"]):
        assert oracle.region(s, soa, c).tobytes() == np.ascontiguousarray(recs[name]).tobytes()


@pytest.mark.parametrize("n", [0, 3, 500])
def test_jagged_round_trip_canonical(n):
    s, d = _tracks(n, 4)
    aos = oracle.pack(s, d, "aos")
    soa = oracle.convert(s, aos, "soa", m=d["m"])
    back = oracle.convert(s, soa, "aos", m=d["m"])
    assert back.base.tobytes() == aos.base.tobytes()
    assert back.pool[: d["m"] * 8].tobytes() == aos.pool[: d["m"] * 8].tobytes()
    # canonical pool: begin == offset, length == difference
    recs = np.frombuffer(back.base[: n * 24].tobytes(), struct_dtype(datagen.TRACKS), count=n)
    off = np.concatenate([[0], np.cumsum(d["lengths"].astype(np.int64))])
    assert recs["hits_begin"].tolist() == off[:-1].tolist()
    assert recs["hits_length"].tolist() == d["lengths"].tolist()


def test_jagged_empty_children_and_u64_offsets():
    desc = [("a", "u8", 1), ("v", "jagged", "u64", [("x", "f64", 1)])]
    s = oracle.Schema(desc)
    d = datagen.jagged_random(desc, 50, 3, mean_len=0.0)
    assert d["m"] == 0
    aos = oracle.pack(s, d, "aos")
    soa = oracle.convert(s, aos, "soa", m=0)
    assert oracle.region(s, soa, s.ncols).view(np.uint64).tolist() == [0] * 51


def test_u32_offset_overflow_is_reported():
    s = oracle.Schema(datagen.TRACKS)
    n = 3
    recs = np.zeros(n, struct_dtype(datagen.TRACKS))
    recs["hits_length"] = 2**31
    recs["hits_begin"] = 0
    raw = np.frombuffer(recs.tobytes(), np.uint8).copy()
    pool = np.zeros(8, np.uint8)  # never read: the prefix sum fails first
    src = oracle.Side("aos", n, 2**32, base=raw, pool=pool)
    dst = oracle.alloc(s, "soa", n, 0)
    st, _ = oracle.convert_into(s, src, dst)
    assert st == oracle.EOVERFLOW


def test_bad_begin_and_small_capacity_rejected():
    s, d = _tracks(20, 6)
    aos = oracle.pack(s, d, "aos")
    bad = oracle.Side("aos", 20, d["m"] - 1, base=aos.base, pool=aos.pool)
    assert oracle.convert_into(s, bad, oracle.alloc(s, "soa", 20, d["m"]))[0] == oracle.EINVAL
    small = oracle.alloc(s, "soa", 20, d["m"] - 1)
    assert oracle.convert_into(s, aos, small)[0] == oracle.ESIZE


# -------------------------------------------------------------- brute force

DTS = ["u8", "u16", "u32", "u64", "f32", "f64"]
FIELD_TYPES = [(dt, e) for dt in DTS for e in (1, 3)]


def _small_schemas():
    out = []
    for k in (1, 2):
        for combo in itertools.product(FIELD_TYPES, repeat=k):
            out.append([("f%d" % i, dt, e) for i, (dt, e) in enumerate(combo)])
    rng = np.random.default_rng(0)
    for _ in range(60):
        idx = rng.integers(0, len(FIELD_TYPES), 3)
        out.append([("f%d" % i, *FIELD_TYPES[j]) for i, j in enumerate(idx)])
    return out


def _unique_bytes(s, n):
    """AoS bytes where field byte k holds (k mod 251) + 1 and padding is 0."""
    raw = np.zeros(max(1, n * s.stride), np.uint8)
    k = 0
    for i in range(n):
        for c in range(s.ncols):
            o = i * s.stride + s.col_aos_off[c]
            for b in range(s.col_size[c]):
                raw[o + b] = (k % 251) + 1
                k += 1
    return raw


@pytest.mark.parametrize("desc", _small_schemas(), ids=lambda d: "-".join("%s%d" % (m[1], m[2]) for m in d))
def test_brute_force_small_schemas(desc):
    s = oracle.Schema(desc)
    dt = struct_dtype(desc)
    assert s.stride == dt.itemsize
    for n in (0, 1, 2, 3, 7, 8, 9):
        raw = _unique_bytes(s, n)
        src = oracle.Side("aos", n, base=raw)
        want = aos_columns(desc, raw, n)
        soa = oracle.convert(s, src, "soa")
        for c in range(s.ncols):
            assert oracle.region(s, soa, c).tobytes() == want[c].tobytes()
        for B in (1, 2, 4, 8):
            blk = oracle.convert(s, src, "aosoa", B)
            cols, blocks = aosoa_columns(desc, blk.base, n, B)
            ref = np.zeros(len(blocks), block_dtype(desc, B))
            for c in range(s.ncols):
                assert cols[c].tobytes() == want[c].tobytes()
                fill_block_column(ref, c, want[c], n)
            assert blk.base[: ref.nbytes].tobytes() == ref.tobytes()
            back = oracle.convert(s, blk, "aos")
            assert back.base[: n * s.stride].tobytes() == raw[: n * s.stride].tobytes()
        # no byte lost or duplicated: the multiset of data bytes is preserved
        got = np.concatenate([oracle.region(s, soa, c) for c in range(s.ncols)]) if n else np.zeros(0, np.uint8)
        assert sorted(got.tolist()) == sorted(raw[raw != 0].tolist())


# ------------------------------------------------ jagged parents in AoSoA(B)

@pytest.mark.parametrize("B", [1, 2, 4, 8, 32, 128])
@pytest.mark.parametrize("n", [0, 1, 2, 3, 7, 8, 9, 300])
def test_jagged_aosoa_regions_and_round_trips(n, B):
    """A jagged AoSoA(B) side is the AoSoA(B) blocks of the parent columns,
    then the offsets and the child columns (each region 128-byte aligned).
    Pinned by: the blocks equal the AoSoA(B) conversion of a schema of the
    parent fields alone; the offsets equal the prefix sum of the lengths;
    the child regions equal the SoA side's; AoS -> AoSoA(B) -> AoS, SoA ->
    AoSoA(B) -> SoA and AoS -> AoSoA(B) -> SoA reproduce the direct
    results byte for byte."""
    s, d = _tracks(n, 12 + B, mean_len=2.0)
    aos = oracle.pack(s, d, "aos")
    soa = oracle.convert(s, aos, "soa", m=d["m"])
    blk = oracle.convert(s, aos, "aosoa", B, m=d["m"])
    assert blk.written == d["m"]
    # region placement
    for r in range(1 + 1 + 2):
        assert s.fm_region_start("aosoa", B, n, d["m"], r) % 128 == 0
    # blocks: the parent columns alone, as a non-jagged AoSoA(B)
    parents = oracle.Schema([("pt", "f32", 1), ("eta", "f32", 1), ("label", "i32", 1)])
    p_soa = oracle.Side("soa", n, 0, cols=[oracle.region(s, soa, c).copy() for c in range(3)],
                        base=np.zeros(1, np.uint8))
    p_blk = oracle.convert(parents, p_soa, "aosoa", B)
    assert oracle.region(s, blk, 0).tobytes() == p_blk.base[: parents.base_bytes("aosoa", B, n)].tobytes()
    # the offsets follow the parents' blocks directly (the next multiple of
    # 128 after the blocks of the parent-only schema)
    assert s.fm_region_start("aosoa", B, n, d["m"], 1) == (parents.base_bytes("aosoa", B, n) + 127) // 128 * 128
    # offsets and children as on the SoA side
    for r in range(3):
        assert oracle.region(s, blk, 1 + r).tobytes() == oracle.region(s, soa, s.ncols + r).tobytes()
    off = oracle.region(s, blk, 1).view(np.uint32).astype(np.int64)
    assert off.tolist() == np.concatenate([[0], np.cumsum(d["lengths"].astype(np.int64))]).tolist()
    # round trips and paths through AoSoA(B)
    back = oracle.convert(s, blk, "aos", m=d["m"])
    assert back.base.tobytes() == aos.base.tobytes()
    assert back.pool[: d["m"] * 8].tobytes() == aos.pool[: d["m"] * 8].tobytes()
    assert oracle.convert(s, blk, "soa", m=d["m"]).base.tobytes() == soa.base.tobytes()
    assert oracle.convert(s, soa, "aosoa", B, m=d["m"]).base.tobytes() == blk.base.tobytes()
    other = 32 if B != 32 else 8
    assert oracle.convert(s, oracle.convert(s, blk, "aosoa", other, m=d["m"]), "aosoa", B,
                          m=d["m"]).base.tobytes() == blk.base.tobytes()


def test_jagged_aosoa_tail_slots_and_gaps_are_zero():
    """Every byte of a jagged AoSoA side that holds no value is zero: the
    unused slots of the last block and the bytes between regions."""
    n, B = 37, 32
    s, d = _tracks(n, 5, raw=True)
    aos = oracle.pack(s, d, "aos")
    blk = oracle.convert(s, aos, "aosoa", B, m=d["m"])
    mask = np.zeros(blk.base.size, bool)
    for r in range(4):
        st = s.fm_region_start("aosoa", B, n, d["m"], r)
        mask[st: st + oracle.region(s, blk, r).size] = True
    assert not blk.base[~mask].any()
    blocks = oracle.region(s, blk, 0).reshape(2, -1)
    for c in range(3):  # slots 37 - 32 = 5 .. 31 of the second block
        start = s.aosoa_col_start(B, c)
        col = blocks[1, start: start + B * 4].reshape(B, 4)
        assert not col[n - B:].any()


# ------------------------------------------- size-changing operations (Sec. VI-B)

from oracle import collection as oc  # noqa: E402

ONE = [("v", "u32", 1)]
JAG = [("p", "u16", 1), ("k", "jagged", "u32", [("x", "u8", 1)])]


def _one(vals):
    return {"n": len(vals), "columns": [np.array(vals, np.uint32)]}


def _jag(p, lengths, kids):
    return {"n": len(p), "columns": [np.array(p, np.uint16)], "lengths": np.array(lengths, np.uint32),
            "children": [np.array(kids, np.uint8)], "m": len(kids)}


def test_collection_ops_worked_examples():
    """Hand-written results of the vector-like operations."""
    d = _one([10, 20, 30])
    assert oc.erase(d, 1, 1)["columns"][0].tolist() == [10, 30]
    assert oc.insert(d, 1, _one([99]))["columns"][0].tolist() == [10, 99, 20, 30]
    assert oc.insert(d, 3, _one([7, 8]))["columns"][0].tolist() == [10, 20, 30, 7, 8]
    assert oc.resize(d, 5)["columns"][0].tolist() == [10, 20, 30, 0, 0]
    assert oc.resize(d, 1)["columns"][0].tolist() == [10]
    assert oc.take(d, 1, 2)["columns"][0].tolist() == [20, 30]
    j = _jag([1, 2, 3], [2, 0, 1], [5, 6, 7])
    e = oc.erase(j, 0, 1)
    assert (e["n"], e["m"], e["lengths"].tolist(), e["children"][0].tolist()) == (2, 1, [0, 1], [7])
    e = oc.erase(j, 1, 1)   # an object without children
    assert (e["m"], e["lengths"].tolist(), e["children"][0].tolist()) == (3, [2, 1], [5, 6, 7])
    i = oc.insert(j, 1, _jag([9], [2], [8, 9]))
    assert i["columns"][0].tolist() == [1, 9, 2, 3]
    assert (i["m"], i["lengths"].tolist(), i["children"][0].tolist()) == (5, [2, 2, 0, 1], [5, 6, 8, 9, 7])
    r = oc.resize(j, 4)
    assert (r["lengths"].tolist(), r["children"][0].tolist(), r["columns"][0].tolist()) == \
        ([2, 0, 1, 0], [5, 6, 7], [1, 2, 3, 0])


@pytest.mark.parametrize("name,n", [("cells", 0), ("cells", 57), ("tracks", 41)])
def test_collection_ops_identities(name, n):
    """Erase and re-insert, grow and shrink, split and rejoin give back the
    original, and the laid-out SoA of an erased collection is the SoA with
    the erased rows (and children) cut out of every region."""
    s = oracle.Schema(datagen.WORKLOAD_SCHEMAS[name])
    d = datagen.workload(name, n, 5)
    rng = np.random.default_rng(1)
    for _ in range(5):
        f = int(rng.integers(0, n + 1))
        c = int(rng.integers(0, n - f + 1))
        back = oc.insert(oc.erase(d, f, c), f, oc.take(d, f, c))
        assert oracle.pack(s, back, "soa").base.tobytes() == oracle.pack(s, d, "soa").base.tobytes()
        assert oracle.pack(s, oc.resize(oc.resize(d, n + 9), n), "aos").base.tobytes() == \
            oracle.pack(s, d, "aos").base.tobytes()
        # laid out: each region is the concatenation of the kept rows
        full, cut = oracle.pack(s, d, "soa"), oracle.pack(s, oc.erase(d, f, c), "soa")
        for r in range(s.ncols):
            col = oracle.region(s, full, r)
            sz = col.size // max(n, 1) if n else 0
            want = np.concatenate([col[: f * sz], col[(f + c) * sz:]]) if n else col
            assert oracle.region(s, cut, r).tobytes() == want.tobytes()
        if s.has_jagged:
            off = oracle.region(s, full, s.ncols).view(np.uint32).astype(np.int64)
            a, b = int(off[f]), int(off[f + c])
            for r in range(s.ncols + 1, s.ncols + 1 + len(d["children"])):
                kid = oracle.region(s, full, r)
                ksz = kid.size // max(d["m"], 1)
                want = np.concatenate([kid[: a * ksz], kid[b * ksz:]])
                assert oracle.region(s, cut, r).tobytes() == want.tobytes()
            coff = oracle.region(s, cut, s.ncols).view(np.uint32).astype(np.int64)
            want = np.concatenate([off[:f], off[f + c:] - (b - a)])
            assert coff.tolist() == want.tolist()
    empty = oc.erase(d, 0, n)
    assert empty["n"] == 0 and (not s.has_jagged or empty["m"] == 0)


# ------------------------------------------- interleaved array properties
# An array property declared interleaved is stored field-major as ONE N x E
# array (Sec. V, array property, its single-array interface): record i's
# element k at row i, position k.  numpy's row-major subarray fields are
# that array, and numpy's aligned structs with (B, E) members are the AoSoA
# block; AoS is unchanged (the C array inside the record).

from np_layout import leaf_kinds, storage_block_dtype, storage_values  # noqa: E402

INTERLEAVED = [("id", "u32", 1), ("pos", "f32", 3, "interleaved"), ("flag", "u8", 1),
               ("w", "u16", 4, "interleaved"), ("k", "u64", 2, "interleaved"),
               ("c", "u8", 3, "interleaved"), ("plain", "u16", 2)]
IL_SCHEMAS = {"mixed": INTERLEAVED,
              "only": [("v", "f64", 3, "interleaved")],
              "grouped": [("a", "u8", 1), ("g", "group", [("x", "u32", 3, "interleaved"), ("y", "u8", 1)]),
                          ("b", "u16", 4, "interleaved")]}


def _storage_first_cols(desc):
    """Flattened index of the first column of every storage column."""
    out, c = [], 0
    for dt, e, inter in leaf_kinds(desc):
        if inter:
            out.append(c)
            c += e
        else:
            for _ in range(e):
                out.append(c)
                c += 1
    return out


@pytest.mark.parametrize("name", list(IL_SCHEMAS))
def test_interleaved_aos_is_the_c_array(name):
    desc = IL_SCHEMAS[name]
    s = oracle.Schema(desc)
    dt = struct_dtype(desc)
    assert s.stride == dt.itemsize
    for n in (0, 1, 9, 300):
        d = values_for(desc, n, 31)
        aos = oracle.pack(s, d, "aos")
        assert aos.base[: n * s.stride].tobytes() == aos_from_values(desc, d["columns"], n).tobytes()


@pytest.mark.parametrize("name", list(IL_SCHEMAS))
@pytest.mark.parametrize("n", [0, 1, 5, 129, 1000])
def test_interleaved_soa_is_the_row_major_array(name, n):
    desc = IL_SCHEMAS[name]
    s = oracle.Schema(desc)
    ref = aos_from_values(desc, values_for(desc, n, 7)["columns"], n)
    raw = np.frombuffer(ref.tobytes(), np.uint8).copy() if n else np.zeros(1, np.uint8)
    soa = oracle.convert(s, oracle.Side("aos", n, base=raw), "soa")
    arrs = storage_values(desc, [get for get in _numpy_leaves(desc, ref)])
    firsts = _storage_first_cols(desc)
    assert s.nstore == len(arrs)
    mask = np.ones(soa.base.size, bool)
    for q, (c, a) in enumerate(zip(firsts, arrs)):
        st = s.soa_region_start(n, 0, c)
        nb = a.nbytes
        assert st % 128 == 0
        assert soa.base[st:st + nb].tobytes() == a.tobytes(), "storage column %d" % q
        mask[st:st + nb] = False
    assert not soa.base[mask].any()
    # the other columns of an interleaved array start at their element
    for c in range(s.ncols):
        assert s.soa_region_start(n, 0, c) == s.soa_region_start(n, 0, firsts[s.col_store[c]]) + s.col_sub[c]


def _numpy_leaves(desc, arr):
    from np_layout import leaf_paths, get_leaf
    return [np.asarray(get_leaf(arr, p)) for p, _, _ in leaf_paths(desc)]


@pytest.mark.parametrize("name", list(IL_SCHEMAS))
@pytest.mark.parametrize("B", [1, 3, 8, 32])
@pytest.mark.parametrize("n", [0, 1, 31, 33, 300])
def test_interleaved_aosoa_matches_numpy_block_struct(name, B, n):
    desc = IL_SCHEMAS[name]
    s = oracle.Schema(desc)
    d = values_for(desc, n, 13)
    bd = storage_block_dtype(desc, B)
    assert s.aosoa_block_bytes(B) == bd.itemsize
    out = oracle.pack(s, d, "aosoa", B)
    nb = (n + B - 1) // B
    ref = np.zeros(nb, bd)
    for q, v in enumerate(storage_values(desc, d["columns"])):
        fld = ref["s%d" % q]
        full = np.zeros((nb * B,) + v.shape[1:], fld.dtype)
        full[:n] = v.view(fld.dtype) if v.dtype != fld.dtype else v
        fld[...] = full.reshape(fld.shape)
    assert out.base[: ref.nbytes].tobytes() == ref.tobytes()


@pytest.mark.parametrize("name", list(IL_SCHEMAS))
@pytest.mark.parametrize("n", [0, 1, 100, 4097])
def test_interleaved_round_trips(name, n):
    desc = IL_SCHEMAS[name]
    s = oracle.Schema(desc)
    aos = oracle.pack(s, values_for(desc, n, 17), "aos")
    soa = oracle.convert(s, aos, "soa")
    assert oracle.convert(s, soa, "aos").base.tobytes() == aos.base.tobytes()
    b = oracle.convert(s, oracle.convert(s, oracle.convert(s, aos, "aosoa", 32), "soa"), "aos")
    assert b.base.tobytes() == aos.base.tobytes()
    c = oracle.convert(s, oracle.convert(s, oracle.convert(s, soa, "aosoa", 32), "aosoa", 128), "soa")
    assert c.base.tobytes() == soa.base.tobytes()


def test_interleaved_special_cases():
    # extent 1: interleaving changes nothing, in any layout
    n = 50
    a, b = [("v", "u32", 1), ("t", "u8", 1)], [("v", "u32", 1, "interleaved"), ("t", "u8", 1)]
    sa, sb = oracle.Schema(a), oracle.Schema(b)
    d = values_for(a, n, 3)
    for kind, B in [("aos", 0), ("soa", 0), ("aosoa", 8)]:
        assert oracle.pack(sa, d, kind, B).base.tobytes() == oracle.pack(sb, d, kind, B).base.tobytes()
    # a single interleaved array of a record without padding: the SoA array
    # is the AoS buffer itself
    one = [("v", "u16", 5, "interleaved")]
    so = oracle.Schema(one)
    d = values_for(one, n, 4)
    aos = oracle.pack(so, d, "aos")
    soa = oracle.convert(so, aos, "soa")
    assert soa.base[: n * 10].tobytes() == aos.base[: n * 10].tobytes()
    # one block holding every record equals the single-block SoA of B records
    B = 64
    blk = oracle.convert(so, aos, "aosoa", B)
    soa_b = oracle.convert(so, oracle.pack(so, values_for(one, B, 4), "aos"), "soa")
    assert blk.base[: n * 10].tobytes() == soa_b.base[: n * 10].tobytes()
    assert not blk.base[n * 10: B * 10].any()


IL_FIELD_TYPES = [(dt, e, "interleaved") for dt in DTS for e in (2, 3)]


def _small_interleaved_schemas():
    rng = np.random.default_rng(5)
    out = [[("f0",) + t] for t in IL_FIELD_TYPES]
    pool = FIELD_TYPES + IL_FIELD_TYPES
    for _ in range(60):
        idx = rng.integers(0, len(pool), 3)
        out.append([("f%d" % i,) + tuple(pool[j]) for i, j in enumerate(idx)])
    return out


@pytest.mark.parametrize("desc", _small_interleaved_schemas(), ids=lambda d: "-".join("%s%d%s" % (
    m[1], m[2], "i" if len(m) > 3 else "") for m in d))
def test_brute_force_interleaved_schemas(desc):
    """Unique field bytes through SoA and AoSoA(B) and back: every storage
    column equals numpy's (row-major rows for interleaved arrays), no byte
    is lost, duplicated or misplaced, and the padding is zero."""
    s = oracle.Schema(desc)
    dt = struct_dtype(desc)
    assert s.stride == dt.itemsize
    for n in (0, 1, 2, 3, 7, 8, 9):
        raw = _unique_bytes(s, n)
        arr = np.frombuffer(raw[: n * s.stride].tobytes(), dt, count=n)
        arrs = storage_values(desc, _numpy_leaves(desc, arr))
        src = oracle.Side("aos", n, base=raw)
        soa = oracle.convert(s, src, "soa")
        for c, a in zip(_storage_first_cols(desc), arrs):
            st = s.soa_region_start(n, 0, c)
            assert soa.base[st:st + a.nbytes].tobytes() == a.tobytes()
        assert oracle.convert(s, soa, "aos").base[: n * s.stride].tobytes() == raw[: n * s.stride].tobytes()
        for B in (1, 2, 4, 8):
            blk = oracle.convert(s, src, "aosoa", B)
            bd = storage_block_dtype(desc, B)
            nb = (n + B - 1) // B
            blocks = np.frombuffer(blk.base[: nb * bd.itemsize].tobytes(), bd, count=nb)
            for q, a in enumerate(arrs):
                got = blocks["s%d" % q].reshape((nb * B,) + a.shape[1:])
                assert got[:n].tobytes() == a.tobytes()
                assert not got[n:].view(np.uint8).any()
            assert oracle.convert(s, blk, "aos").base[: n * s.stride].tobytes() == raw[: n * s.stride].tobytes()


# --------------------------------------------------- nested jagged members
# A jagged member may nest once (the children are a collection described by
# properties, Sec. V): every hit of a track holds its own list of samples.
# The pins: numpy's C structs for both record levels, the offsets invariants
# at both levels, round trips, a zero-length special case, and a brute-force
# walk over shuffled pools at both levels on tiny inputs.

def _nested(n, seed, raw=False):
    s = oracle.Schema(datagen.TRACKS_NESTED)
    return s, datagen.workload("tracks_nested", n, seed, raw=raw)


def test_nested_strides_match_numpy():
    s = oracle.Schema(datagen.TRACKS_NESTED)
    child_desc = datagen.jagged_member(datagen.TRACKS_NESTED)[2]
    grand_desc = datagen.jagged_member(child_desc)[2]
    assert s.stride == struct_dtype(datagen.TRACKS_NESTED).itemsize
    assert s.child.stride == struct_dtype(child_desc).itemsize == 24
    assert (s.child.len_off, s.child.begin_off) == (8, 16)
    assert s.child.child.stride == struct_dtype(grand_desc).itemsize == 4


@pytest.mark.parametrize("n", [0, 1, 17, 1000])
def test_nested_soa_columns_and_offsets_invariants(n):
    s, d = _nested(n, 3)
    aos = oracle.pack(s, d, "aos")
    soa = oracle.convert(s, aos, "soa")
    m, m2 = d["m"], d["m2"]
    base = soa.base
    # parents
    for c, v in enumerate(d["columns"]):
        st = s.soa_region_start(n, m, c, m2)
        assert base[st: st + v.nbytes].tobytes() == v.tobytes()
    # offsets at both levels: exclusive scans ending at the totals
    st = s.soa_region_start(n, m, s.ncols, m2)
    off0 = base[st: st + 4 * (n + 1)].view("<u4")
    assert off0.tolist() == np.concatenate([[0], np.cumsum(d["lengths"].astype(np.uint64))]).tolist()
    assert int(off0[-1]) == m
    r = s.ncols + 1
    for c, v in enumerate(d["children"]):
        st = s.soa_region_start(n, m, r + c, m2)
        assert base[st: st + v.nbytes].tobytes() == v.tobytes()
    st = s.soa_region_start(n, m, r + s.child.ncols, m2)
    off1 = base[st: st + 4 * (m + 1)].view("<u4")
    assert off1.tolist() == np.concatenate([[0], np.cumsum(d["child_lengths"].astype(np.uint64))]).tolist()
    assert int(off1[-1]) == m2
    for g, v in enumerate(d["grandchildren"]):
        st = s.soa_region_start(n, m, r + s.child.ncols + 1 + g, m2)
        assert st % 128 == 0
        assert base[st: st + v.nbytes].tobytes() == v.tobytes()


@pytest.mark.parametrize("n", [0, 1, 300])
def test_nested_round_trips(n):
    s, d = _nested(n, 5, raw=True)
    aos = oracle.pack(s, d, "aos")
    soa = oracle.convert(s, aos, "soa")
    back = oracle.convert(s, soa, "aos")
    assert back.base.tobytes() == aos.base.tobytes()
    assert back.pool.tobytes() == aos.pool.tobytes()
    assert back.gpool.tobytes() == aos.gpool.tobytes()
    for B in (1, 3, 32):
        blk = oracle.convert(s, aos, "aosoa", B)
        again = oracle.convert(s, blk, "aos")
        assert again.base.tobytes() == aos.base.tobytes() and again.gpool.tobytes() == aos.gpool.tobytes()
        assert oracle.convert(s, blk, "soa").base.tobytes() == soa.base.tobytes()
        assert oracle.convert(s, soa, "aosoa", B).base.tobytes() == blk.base.tobytes()


def test_nested_with_no_grandchildren_is_the_flat_layout_plus_zero_offsets():
    n = 200
    s, d = _nested(n, 9)
    d["child_lengths"] = np.zeros(d["m"], np.uint32)
    d["grandchildren"] = [g[:0] for g in d["grandchildren"]]
    d["m2"] = 0
    flat = oracle.Schema([m if m[1] != "jagged" else (m[0], m[1], m[2], m[3][:2]) for m in datagen.TRACKS_NESTED])
    soa = oracle.convert(s, oracle.pack(s, d, "aos"), "soa")
    ref = oracle.pack(flat, d, "soa")
    head = flat.base_bytes("soa", 0, n, d["m"])
    assert soa.base[:head].tobytes() == ref.base[:head].tobytes()
    st = s.soa_region_start(n, d["m"], s.ncols + 1 + s.child.ncols, 0)
    assert st == head and not soa.base[st:].any()


def _jagged_path(desc):
    """Group names leading to the jagged member, then its name."""
    for m in desc:
        if m[1] == "jagged":
            return [m[0]]
        if m[1] == "group":
            p = _jagged_path(m[2])
            if p:
                return [m[0]] + p
    return None


def _at(rec, path, suffix):
    for g in path[:-1]:
        rec = rec[g]
    return rec[path[-1] + suffix]


def _walk_nested(desc, n, recs, pool, gpool):
    """Brute force: the canonical child and grandchild sequences, walking
    numpy records parent by parent, child by child."""
    jn, _, cdesc = datagen.jagged_member(desc)
    gn, _, gdesc = datagen.jagged_member(cdesc)
    jp, gp = _jagged_path(desc), _jagged_path(cdesc)
    pd, cd, gd = struct_dtype(desc), struct_dtype(cdesc), struct_dtype(gdesc)
    P = np.frombuffer(recs[: n * pd.itemsize].tobytes(), pd, count=n)
    C = np.frombuffer(pool.tobytes(), cd, count=pool.size // cd.itemsize)
    G = np.frombuffer(gpool.tobytes(), gd, count=gpool.size // gd.itemsize)
    kids, grand, off0, off1 = [], [], [0], [0]
    for i in range(n):
        b, L = int(_at(P[i], jp, "_begin")), int(_at(P[i], jp, "_length"))
        for k in range(L):
            c = C[b + k]
            kids.append(c)
            b1, L1 = int(_at(c, gp, "_begin")), int(_at(c, gp, "_length"))
            grand += [G[b1 + q] for q in range(L1)]
            off1.append(off1[-1] + L1)
        off0.append(off0[-1] + L)
    return kids, grand, off0, off1


NESTED_SMALL = [
    [("a", "u8", 1), ("v", "jagged", "u32", [("x", "u16", 1), ("w", "jagged", "u32", [("y", "u8", 1)])])],
    [("v", "jagged", "u64", [("w", "jagged", "u32", [("y", "u64", 1), ("z", "u8", 3)]), ("x", "f32", 1)]),
     ("b", "u32", 2)],
    [("g", "group", [("p", "f64", 1), ("v", "jagged", "u32", [("x", "u8", 2, "interleaved"),
                                                            ("w", "jagged", "u64", [("y", "u16", 1)])])])],
]


from nested_util import shuffle_runs as _shuffle_runs  # noqa: E402


@pytest.mark.parametrize("k", range(len(NESTED_SMALL)))
def test_brute_force_nested_shuffled_pools(k):
    """Tiny nested collections whose pools are shuffled at both levels (runs
    in random order, a free slot before each): the SoA output equals a
    walk over the numpy records, parent by parent and child by child, and
    converts back to the same values."""
    from np_layout import leaf_paths, get_leaf
    desc = NESTED_SMALL[k]
    cdesc = datagen.jagged_member(desc)[2]
    gdesc = datagen.jagged_member(cdesc)[2]
    s = oracle.Schema(desc)
    cs, gs = s.child.stride, s.child.child.stride
    for n in (0, 1, 2, 5, 9):
        d = datagen.jagged_random(desc, n, 100 + n, mean_len=2.0, max_len=4)
        aos = oracle.pack(s, d, "aos")
        m, m2 = d["m"], d["m2"]
        rng = np.random.default_rng(7 * n + k)
        kids = aos.pool[: max(1, m * cs)].copy()
        gpool = _shuffle_runs(kids, m, cs, s.child.len_off, s.child.begin_off, aos.gpool, gs, rng.permutation(m), 1)
        recs = aos.base.copy()
        pool = _shuffle_runs(recs, n, s.stride, s.len_off, s.begin_off, kids, cs, rng.permutation(n), 1)
        src = oracle.Side("aos", n, (pool.size // cs) if m else 0, base=recs, pool=pool, gpool=gpool,
                          m2=(gpool.size // gs) if m2 else 0)
        soa = oracle.convert(s, src, "soa", m=m, m2=m2)
        assert soa.written == m
        kid_recs, grand, off0, off1 = _walk_nested(desc, n, recs, pool, gpool)
        base = soa.base
        st = s.soa_region_start(n, m, s.ncols, m2)
        assert base[st: st + s.off_size * (n + 1)].view("<u%d" % s.off_size).tolist() == off0
        st = s.soa_region_start(n, m, s.ncols + 1 + s.child.ncols, m2)
        o1 = s.child.off_size
        assert base[st: st + o1 * (m + 1)].view("<u%d" % o1).tolist() == off1
        for level, (recs_l, ldesc, first, lsch) in enumerate(
                [(kid_recs, cdesc, s.ncols + 1, s.child),
                 (grand, gdesc, s.ncols + 2 + s.child.ncols, s.child.child)]):
            col = 0
            for path, _, e in leaf_paths(ldesc):
                for kk in range(e):
                    st = s.soa_region_start(n, m, first + col, m2)
                    es = lsch.col_es[col]
                    for j, rec in enumerate(recs_l):
                        v = np.asarray(get_leaf(rec, path))
                        want = (v if e == 1 else v[kk]).tobytes()
                        assert base[st + j * es: st + j * es + len(want)].tobytes() == want, (level, col, j)
                    col += 1
        # and back: the canonical pools hold the same values in walk order
        back = oracle.convert(s, soa, "aos")
        k2, g2, _, _ = _walk_nested(desc, n, back.base, back.pool, back.gpool)
        strip = lambda r, dd: [np.asarray(get_leaf(r, p)).tobytes() for p, _, _ in leaf_paths(dd)]  # noqa: E731
        assert [strip(r, cdesc) for r in k2] == [strip(r, cdesc) for r in kid_recs]
        assert [strip(r, gdesc) for r in g2] == [strip(r, gdesc) for r in grand]


def test_interleaved_parent_array_with_a_jagged_member():
    """A jagged schema whose parents hold an interleaved array: the parent
    storage columns, then the offsets and the child columns, each where the
    column-counted item index says; numpy rows for the array, cumsum for
    the offsets, round trips through SoA and AoSoA(B)."""
    desc = [("pt", "f32", 1), ("cov", "f32", 3, "interleaved"),
            ("hits", "jagged", "u32", [("index", "u32", 1), ("weight", "f32", 1)])]
    s = oracle.Schema(desc)
    n = 257
    d = datagen.random_columns(desc, n, 6)
    dj = datagen.workload("tracks", n, 7)
    d.update(lengths=dj["lengths"], children=dj["children"], m=dj["m"])
    aos = oracle.pack(s, d, "aos")
    soa = oracle.convert(s, aos, "soa")
    m = d["m"]
    st = s.soa_region_start(n, m, 1)
    assert soa.base[st: st + 12 * n].tobytes() == np.ascontiguousarray(d["columns"][1]).tobytes()
    st = s.soa_region_start(n, m, s.ncols)
    assert soa.base[st: st + 4 * (n + 1)].view("<u4").tolist() == \
        np.concatenate([[0], np.cumsum(d["lengths"].astype(np.uint64))]).tolist()
    for c, v in enumerate(d["children"]):
        st = s.soa_region_start(n, m, s.ncols + 1 + c)
        assert soa.base[st: st + v.nbytes].tobytes() == v.tobytes()
    assert oracle.convert(s, soa, "aos").base.tobytes() == aos.base.tobytes()
    for B in (3, 32):
        assert oracle.convert(s, oracle.convert(s, aos, "aosoa", B), "soa").base.tobytes() == soa.base.tobytes()
