"""GPU parity of interleaved array properties (one field-major N x E array
per property, the array property's single-array interface of Sec. V):
every layout pair, extents 3 and 4 over element sizes 1, 2, 4 and 8,
sizes across tiles with a ragged tail, per-column views, jagged parents
with an interleaved array, and batches, each equal to the oracle's bytes."""
import numpy as np
import pytest

import datagen
import oracle
import paper_2511_04853_b300 as mrn
from gpu_util import dev, dev_dest, garbage, host

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, params=["staged", "direct"])
def conversion_path(request):
    """Every test of this module runs twice: single conversions on the
    TMA-staged kernel wherever it applies (an interleaved array's rows are
    one bulk copy per tile, its elements at slot * row bytes in the tile),
    and on the direct kernel only."""
    mrn.debug_set(3, 1 if request.param == "direct" else 0)
    yield request.param
    mrn.debug_set(3, 0)

DTYPES = {1: "u8", 2: "u16", 4: "f32", 8: "u64"}
PAIRS = [("aos", 0, "soa", 0), ("soa", 0, "aos", 0), ("aos", 0, "aosoa", 32), ("aosoa", 32, "aos", 0),
         ("soa", 0, "aosoa", 5), ("aosoa", 5, "soa", 0), ("aosoa", 32, "aosoa", 128)]
MIXED = [("id", "u32", 1), ("pos", "f32", 3, "interleaved"), ("flag", "u8", 1),
         ("g", "group", [("w", "u16", 4, "interleaved"), ("k", "u64", 2, "interleaved")]),
         ("c", "u8", 3, "interleaved"), ("plain", "u16", 2)]


def one_array(size, E):
    return [("id", "u32", 1), ("a", DTYPES[size], E, "interleaved"), ("t", "u8", 1)]


def check_pair(desc, n, sk, sb, dk, db, seed=1):
    s, o = mrn.Schema(desc), oracle.Schema(desc)
    d = datagen.random_columns(desc, n, seed)
    o_src = oracle.pack(o, d, sk, sb)
    want = oracle.convert(o, o_src, dk, db).base[: s.required_bytes(dk, n, 0, db)]
    dst = dev_dest(s, dk, n, 0, db)
    mrn.convert(mrn.View(s, sk, n, block=sb, base=dev(o_src.base)), dst)
    assert mrn.sync() == mrn.OK
    got = host(dst.tensors[0], want.size)
    assert np.array_equal(got, want), "%s %s%s -> %s%s n=%d" % (desc, sk, sb or "", dk, db or "", n)


@pytest.mark.parametrize("size", [1, 2, 4, 8])
@pytest.mark.parametrize("E", [3, 4])
@pytest.mark.parametrize("pair", PAIRS)
def test_every_pair_extent_and_size(size, E, pair):
    for n in (1, 1000, 70001):
        check_pair(one_array(size, E), n, *pair, seed=size * 10 + E)


@pytest.mark.parametrize("pair", PAIRS)
def test_wide_rows(pair):
    """Rows of 240 bytes (f32[60]: a staged tile of 32 records) and of
    480 bytes (u64[60]: 32 records exceed a stage, the direct kernel
    only)."""
    for E, size, n in ((60, 4, 1000), (60, 8, 300)):
        check_pair(one_array(size, E), n, *pair, seed=E)


@pytest.mark.parametrize("pair", PAIRS)
@pytest.mark.parametrize("n", [0, 33, 4097, 200003])
def test_mixed_schema_all_pairs(pair, n):
    check_pair(MIXED, n, *pair, seed=n % 97)


def test_per_column_views_and_consecutive_element_rule():
    """A SoA view with per-column pointers: column k of an interleaved array
    points at element k of the array's first row; results equal the
    oracle's, and pointers that are not consecutive elements are refused."""
    desc = MIXED
    s, o = mrn.Schema(desc), oracle.Schema(desc)
    n = 5001
    d = datagen.random_columns(desc, n, 4)
    o_aos = oracle.pack(o, d, "aos")
    want = oracle.convert(o, o_aos, "soa")
    block = garbage(s.required_bytes("soa", n))
    cols = [block.data_ptr() + s.soa_region_offset(n, 0, c) for c in range(s.ncols)]
    mrn.convert(mrn.View(s, "aos", n, base=dev(o_aos.base)), mrn.View(s, "soa", n, columns=cols))
    assert mrn.sync() == mrn.OK
    got = host(block)
    for c in range(s.ncols):
        st = s.soa_region_offset(n, 0, c)
        es = s.columns[c]["fm_stride"]
        assert st == o.soa_region_start(n, 0, c)
        assert np.array_equal(got[st: st + (n - 1) * es + s.columns[c]["size"]],
                              want.base[st: st + (n - 1) * es + s.columns[c]["size"]]), "column %d" % c
    bad = list(cols)
    k = next(c for c in range(s.ncols) if s.columns[c]["fm_stride"] != s.columns[c]["size"]) + 1
    bad[k] += s.columns[k]["size"]
    st = mrn.convert_status(mrn.View(s, "aos", n, base=dev(o_aos.base)), mrn.View(s, "soa", n, columns=bad))
    assert st == mrn.EINVAL


def test_jagged_parents_with_an_interleaved_array():
    desc = [("pt", "f32", 1), ("cov", "f32", 3, "interleaved"),
            ("hits", "jagged", "u32", [("index", "u32", 1), ("weight", "f32", 1)])]
    s, o = mrn.Schema(desc), oracle.Schema(desc)
    for n in (1, 3000, 70001):
        d = datagen.random_columns(desc[:2], n, 6)
        dj = datagen.workload("tracks", n, 7)
        d = {"n": n, "columns": d["columns"], "lengths": dj["lengths"], "children": dj["children"], "m": dj["m"]}
        o_aos = oracle.pack(o, d, "aos")
        for dk, db in (("soa", 0), ("aosoa", 32)):
            want = oracle.convert(o, o_aos, dk, db, m=d["m"])
            dst = dev_dest(s, dk, n, d["m"], db)
            src = mrn.View(s, "aos", n, base=dev(o_aos.base), child_pool=dev(o_aos.pool), m=d["m"])
            mrn.convert(src, dst)
            assert mrn.sync() == mrn.OK
            assert np.array_equal(host(dst.tensors[0], want.base.size), want.base), (n, dk)
            back = dev_dest(s, "aos", n, d["m"])
            mrn.convert(mrn.View(s, dk, n, block=db, base=dst.tensors[0], m=d["m"]), back)
            assert mrn.sync() == mrn.OK
            assert np.array_equal(host(back.tensors[0], n * o.stride), o_aos.base[: n * o.stride])
            assert np.array_equal(host(back.tensors[1], d["m"] * 8), o_aos.pool[: d["m"] * 8])


def test_batch_with_interleaved_jobs():
    pairs, checks = [], []
    for j, (desc, n, sk, sb, dk, db) in enumerate([(MIXED, 20000, "aos", 0, "soa", 0),
                                                   (one_array(2, 3), 7777, "aos", 0, "aosoa", 128),
                                                   (one_array(8, 4), 513, "soa", 0, "aos", 0),
                                                   (datagen.CELLS, 30000, "aos", 0, "soa", 0)]):
        s, o = mrn.Schema(desc), oracle.Schema(desc)
        d = datagen.random_columns(desc, n, 40 + j)
        o_src = oracle.pack(o, d, sk, sb)
        want = oracle.convert(o, o_src, dk, db).base
        dst = dev_dest(s, dk, n, 0, db)
        pairs.append((mrn.View(s, sk, n, block=sb, base=dev(o_src.base)), dst))
        checks.append((dst, want))
    for use_graph in (True, False):
        for dst, _ in checks:
            dst.tensors[0].fill_(0xA5)
        b = mrn.Batch(pairs, use_graph=use_graph)
        b.launch()
        assert mrn.sync() == mrn.OK
        for k, (dst, want) in enumerate(checks):
            assert np.array_equal(host(dst.tensors[0], want.size), want), "job %d" % k


def test_transfer_refuses_interleaved():
    import torch
    s = mrn.Schema(one_array(4, 3))
    n = 10
    h = torch.zeros(s.required_bytes("aos", n), dtype=torch.uint8).pin_memory()
    d = garbage(s.required_bytes("soa", n))
    st = mrn.lib().mrn_transfer_convert(mrn.View(s, "aos", n, base=h, mem="pinned").ref,
                                        mrn.View(s, "soa", n, base=d).ref, None, mrn.mrn._stream(None))
    assert st == mrn.EUNSUPPORTED
