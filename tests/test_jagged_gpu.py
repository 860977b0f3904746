"""GPU parity of the jagged path (Sec. V, jagged vector property): the prefix
sum of the sizes and the flattened children must equal the oracle's exactly,
in both directions, for canonical and shuffled child pools; the device-side
checks (offset overflow, child capacity, child indices, bounded look-back
waits) must report their status codes without faulting."""
import numpy as np
import pytest

import datagen
import oracle
import paper_2511_04853_b300 as mrn
from gpu_util import dev, dev_dest, dev_view, garbage, host, torch

pytestmark = pytest.mark.gpu

SPLIT_DEFAULT = 2**63 - 1  # parents from which single conversions run split (debug key 4): never
SMALL_DEFAULT = 250000  # parents up to which fused conversions take 256-parent tiles (debug key 5)


@pytest.fixture(autouse=True, params=["fused", "fused_big", "split", "split_scan"])
def jagged_path(request):
    """Every test of this module runs four times: with jagged AoS ->
    field-major conversions fused (the tiles gather their own children) in
    tiles of 256 parents (the default up to 250,000 parents) and of 1,024,
    and split in the local form (parents with their begins as offsets and
    the pool's checks, pool conversion when canonical, otherwise the whole
    conversion again fused) and in the scan form (debug key 6: scan,
    parents, pool conversion when canonical, gathering pass)."""
    mrn.debug_set(4, 0 if request.param.startswith("split") else -1)
    mrn.debug_set(5, -1 if request.param == "fused_big" else SMALL_DEFAULT)
    mrn.debug_set(6, 1 if request.param == "split_scan" else 0)
    yield request.param
    mrn.debug_set(4, SPLIT_DEFAULT)
    mrn.debug_set(5, SMALL_DEFAULT)
    mrn.debug_set(6, 0)


def tracks(n, seed=2, **kw):
    return mrn.Schema(datagen.TRACKS), oracle.Schema(datagen.TRACKS), datagen.workload("tracks", n, seed, **kw)


def a2s_check(s, o, o_aos, m_cap=None):
    n = o_aos.n
    m = o_aos.m if m_cap is None else m_cap
    o_soa = oracle.convert(o, o_aos, "soa", m=m)
    src = dev_view(s, o_aos, o)
    dst = dev_dest(s, "soa", n, m)
    mrn.convert(src, dst)
    assert mrn.sync() == mrn.OK
    nb = o.base_bytes("soa", 0, n, m)
    got, want = host(dst.tensors[0], nb), o_soa.base[:nb]
    if not np.array_equal(got, want):
        bad = np.nonzero(got != want)[0]
        raise AssertionError("%d bytes differ, first at %d" % (bad.size, bad[0]))
    return o_soa, dst


def test_tracks_100000_both_directions():
    n = 100000
    s, o, d = tracks(n)
    o_aos = oracle.pack(o, d, "aos")
    o_soa, dst = a2s_check(s, o, o_aos)
    off = host(dst.tensors[0])[o.soa_region_start(n, d["m"], 3):][: (n + 1) * 4].view(np.uint32)
    assert off[0] == 0 and off[-1] == d["m"] and (np.diff(off.astype(np.int64)) >= 0).all()
    back = dev_dest(s, "aos", n, d["m"])
    mrn.convert(dst, back)
    assert mrn.sync() == mrn.OK
    assert np.array_equal(host(back.tensors[0], n * 24), o_aos.base[: n * 24])
    assert np.array_equal(host(back.tensors[1], d["m"] * 8), o_aos.pool[: d["m"] * 8])
    assert mrn.jagged_count(dev_view(s, o_aos, o)) == d["m"]


def test_tracks_raw_bits_and_shuffled_pool_with_gaps():
    n = 20000
    s, o, d = tracks(n, seed=5, raw=True)
    o_aos = oracle.pack(o, d, "aos")
    order = np.random.default_rng(9).permutation(n)
    shuffled = oracle.shuffle_pool(o, o_aos, order, gap=2)
    a2s_check(s, o, shuffled, m_cap=d["m"])


def test_stray_empty_begins_and_one_tile_out_of_order():
    """A tile whose children form one run of the pool is gathered without a
    parent lookup; empty parents may carry any begin within the pool without
    breaking the run, and a tile whose runs are out of order (tile 1 here)
    takes the general path.  Both must equal the oracle."""
    n = 4 * 1024 + 17  # four jagged tiles of 1,024 parents and a ragged one
    s, o, d = tracks(n, seed=11, mean_len=2.0)
    o_aos = oracle.pack(o, d, "aos")
    lens = d["lengths"]
    assert (lens == 0).sum() > 50
    order = np.arange(n)
    cand = [i for i in range(1024, 2048) if lens[i] > 0]
    i, j = cand[3], cand[10]
    order[i], order[j] = j, i
    sh = oracle.shuffle_pool(o, o_aos, order, gap=0)
    rng = np.random.default_rng(4)
    recs = sh.base[: n * 24].reshape(n, 24)
    for k in np.nonzero(lens == 0)[0]:
        recs[k, 16:24] = np.array([rng.integers(0, d["m"] + 1)], np.uint64).view(np.uint8)
    a2s_check(s, o, sh, m_cap=d["m"])


@pytest.mark.parametrize("n", [0, 1, 255, 256, 257, 1000, 1023, 1024, 1025, 3073, 5003])
@pytest.mark.parametrize("osz", ["u32", "u64"])
def test_sizes_and_offset_types(n, osz):
    desc = [("a", "u8", 1), ("b", "f64", 1),
            ("v", "jagged", osz, [("x", "u16", 1), ("y", "u8", 3), ("z", "f64", 1)]),
            ("c", "u32", 2)]
    s, o = mrn.Schema(desc), oracle.Schema(desc)
    d = datagen.jagged_random(desc, n, 11 + n, mean_len=3.0, max_len=40)
    o_aos = oracle.pack(o, d, "aos")
    o_soa, dst = a2s_check(s, o, o_aos)
    back = dev_dest(s, "aos", n, d["m"])
    mrn.convert(dst, back)
    assert mrn.sync() == mrn.OK
    assert np.array_equal(host(back.tensors[0], n * o.stride), o_aos.base[: n * o.stride])
    cs = o.child.stride
    assert np.array_equal(host(back.tensors[1], d["m"] * cs), o_aos.pool[: d["m"] * cs])


def test_particle_schema():
    s, o = mrn.Schema(datagen.PARTICLE), oracle.Schema(datagen.PARTICLE)
    n = 3000
    d = datagen.jagged_random(datagen.PARTICLE, n, 4, mean_len=6.0, max_len=25)
    o_aos = oracle.pack(o, d, "aos")
    a2s_check(s, o, o_aos)


def test_long_rows_and_empty_rows():
    """Lengths up to 256 mixed with many zero-length objects."""
    desc = datagen.TRACKS
    s, o = mrn.Schema(desc), oracle.Schema(desc)
    n = 3000
    rng = np.random.default_rng(1)
    lengths = np.where(rng.random(n) < 0.7, 0, rng.integers(200, 257, n)).astype(np.uint32)
    m = int(lengths.sum())
    d = {"columns": [rng.random(n).astype(np.float32), rng.random(n).astype(np.float32),
                     rng.integers(0, 9, n).astype(np.int32)], "n": n, "lengths": lengths,
         "children": [rng.integers(0, 2**32, m, dtype=np.uint64).astype(np.uint32),
                      rng.random(m).astype(np.float32)], "m": m}
    a2s_check(s, o, oracle.pack(o, d, "aos"))


def test_separate_offsets_and_child_columns():
    n = 4000
    s, o, d = tracks(n, seed=3)
    o_aos = oracle.pack(o, d, "aos")
    o_soa = oracle.convert(o, o_aos, "soa", m=d["m"])
    cols = [garbage(n * 4) for _ in range(3)]
    offs = garbage((n + 1) * 4)
    kids = [garbage(d["m"] * 4) for _ in range(2)]
    dst = mrn.View(s, "soa", n, columns=cols, offsets=offs, child_columns=kids, m=d["m"])
    mrn.convert(dev_view(s, o_aos, o), dst)
    assert mrn.sync() == mrn.OK
    for c in range(3):
        assert np.array_equal(host(cols[c]), oracle.region(o, o_soa, c))
    assert np.array_equal(host(offs), oracle.region(o, o_soa, 3))
    for c in range(2):
        assert np.array_equal(host(kids[c]), oracle.region(o, o_soa, 4 + c))


def test_offset_base_shards_concatenate():
    """Two shards converted with offset_base equal the whole collection."""
    n = 6000
    s, o, d = tracks(n, seed=8)
    o_aos = oracle.pack(o, d, "aos")
    o_soa = oracle.convert(o, o_aos, "soa", m=d["m"])
    whole_off = oracle.region(o, o_soa, 3).view(np.uint32)
    half = 2500  # not a multiple of the tile
    lens = d["lengths"]
    m0 = int(lens[:half].sum())
    parts = []
    for lo, hi, base in [(0, half, 0), (half, n, m0)]:
        sub = oracle.Side("aos", hi - lo, o_aos.m, base=o_aos.base[lo * 24: hi * 24].copy(), pool=o_aos.pool)
        mm = int(lens[lo:hi].sum())
        src = mrn.View(s, "aos", hi - lo, base=dev(sub.base), child_pool=dev(o_aos.pool), m=o_aos.m)
        offs = garbage((hi - lo + 1) * 4)
        kids = [garbage(mm * 4) for _ in range(2)]
        cols = [garbage((hi - lo) * 4) for _ in range(3)]
        dst = mrn.View(s, "soa", hi - lo, columns=cols, offsets=offs, child_columns=kids, m=mm,
                       offset_base=base)
        mrn.convert(src, dst)
        assert mrn.sync() == mrn.OK
        parts.append((host(offs).view(np.uint32), [host(k) for k in kids]))
    offs_all = np.concatenate([parts[0][0][:-1], parts[1][0]])
    assert np.array_equal(offs_all, whole_off)
    for c in range(2):
        assert np.array_equal(np.concatenate([parts[0][1][c], parts[1][1][c]]),
                              oracle.region(o, o_soa, 4 + c))


def test_u32_offset_overflow_reported():
    """offset_base close to 2^32: the u32 prefix sum overflows; the kernel
    records MRN_EOVERFLOW (all buffers are real and in bounds)."""
    n = 600
    s, o, d = tracks(n, seed=4)
    o_aos = oracle.pack(o, d, "aos")
    dst = dev_dest(s, "soa", n, d["m"])
    dst.s.offset_base = 2**32 - 100
    mrn.convert(dev_view(s, o_aos, o), dst)
    bits = mrn.sync_bits()
    assert bits & (1 << mrn.EOVERFLOW)


def test_child_capacity_too_small():
    n = 2000
    s, o, d = tracks(n, seed=6)
    o_aos = oracle.pack(o, d, "aos")
    cap = d["m"] // 2
    o_soa = oracle.convert(o, o_aos, "soa", m=d["m"])
    kids = [garbage(cap * 4) for _ in range(2)]
    cols = [garbage(n * 4) for _ in range(3)]
    offs = garbage((n + 1) * 4)
    dst = mrn.View(s, "soa", n, columns=cols, offsets=offs, child_columns=kids, m=cap)
    mrn.convert(dev_view(s, o_aos, o), dst)
    assert mrn.sync() == mrn.ESIZE
    # what fits is still right, and the offsets are complete
    assert np.array_equal(host(offs), oracle.region(o, o_soa, 3))
    for c in range(2):
        assert np.array_equal(host(kids[c]), oracle.region(o, o_soa, 4 + c)[: cap * 4])


def test_child_index_beyond_pool_reported():
    n = 1000
    s, o, d = tracks(n, seed=7)
    o_aos = oracle.pack(o, d, "aos")
    src = mrn.View(s, "aos", n, base=dev(o_aos.base), child_pool=dev(o_aos.pool), m=d["m"] - 5)
    dst = dev_dest(s, "soa", n, d["m"])
    mrn.convert(src, dst)
    assert mrn.sync() == mrn.EINVAL


def test_decreasing_offsets_reported():
    n = 100
    s, o, d = tracks(n, seed=1)
    o_soa = oracle.convert(o, oracle.pack(o, d, "aos"), "soa", m=d["m"])
    base = o_soa.base.copy()
    st = o.soa_region_start(n, d["m"], 3)
    offs = base[st: st + (n + 1) * 4].view(np.uint32)
    offs[50], offs[51] = offs[51], offs[50] + 1000
    src = mrn.View(s, "soa", n, base=dev(base), m=d["m"])
    dst = dev_dest(s, "aos", n, d["m"])
    mrn.convert(src, dst)
    assert mrn.sync() == mrn.EINVAL


def test_lookback_wait_is_bounded(jagged_path):
    """Fault injection on the host side: tile 1 (the split scan's chunk 1)
    never publishes its sum, so the look-back waits of the later ones must
    expire (1 ms bound) and report MRN_ETIMEOUT; the context stays usable
    afterwards.  The local split form looks back only in its fused
    fall-back pass, so there the pool is shuffled (not canonical) to make
    that pass run."""
    n = 4 * 8192  # at least four tiles / scan chunks, at up to 8,192 parents each
    s, o, d = tracks(n, seed=3)
    o_aos = oracle.pack(o, d, "aos")
    if jagged_path == "split":
        o_aos = oracle.shuffle_pool(o, o_aos, np.random.default_rng(4).permutation(n), gap=0)
    try:
        mrn.debug_set(2, 1_000_000)
        mrn.debug_set(1, 1)
        dst = dev_dest(s, "soa", n, d["m"])
        mrn.convert(dev_view(s, o_aos, o), dst)
        assert mrn.sync() == mrn.ETIMEOUT
    finally:
        mrn.debug_set(1, -1)
        mrn.debug_set(2, 2_000_000_000)
    a2s_check(s, o, o_aos)  # normal operation afterwards


def test_equal_jagged_layouts_are_unsupported():
    s = mrn.Schema(datagen.TRACKS)
    buf = garbage(1 << 12)
    a = mrn.View(s, "aosoa", 10, block=32, base=buf, m=1)
    b = mrn.View(s, "aosoa", 10, block=32, base=garbage(1 << 12), m=1)
    assert mrn.convert_status(a, b) == mrn.EUNSUPPORTED


# ---------------------------------------------- jagged parents in AoSoA(B)

def _bytes(view_tensor, n):
    return host(view_tensor, n)


@pytest.mark.parametrize("B", [32, 128, 5])
@pytest.mark.parametrize("n", [0, 1, 511, 512, 513, 1023, 1024, 1025, 2049, 5003])
def test_aos_to_aosoa_and_back(n, B):
    """Jagged AoS -> AoSoA(B): the parent blocks (tail slots zero), the
    offsets and the child columns equal the oracle's, byte for byte, for a
    canonical and a shuffled pool; AoSoA(B) -> AoS gives the canonical AoS
    collection back."""
    s, o, d = tracks(n, seed=40 + B)
    o_aos = oracle.pack(o, d, "aos")
    o_blk = oracle.convert(o, o_aos, "aosoa", B, m=d["m"])
    nb = o.base_bytes("aosoa", B, n, d["m"])
    for src_side in (o_aos, oracle.shuffle_pool(o, o_aos, np.random.default_rng(B).permutation(n), gap=1)):
        dst = dev_dest(s, "aosoa", n, d["m"], B)
        mrn.convert(dev_view(s, src_side, o), dst)
        assert mrn.sync() == mrn.OK
        assert np.array_equal(host(dst.tensors[0], nb), o_blk.base[:nb])
    back = dev_dest(s, "aos", n, d["m"])
    mrn.convert(dev_view(s, o_blk, o), back)
    assert mrn.sync() == mrn.OK
    assert np.array_equal(host(back.tensors[0], n * 24), o_aos.base[: n * 24])
    assert np.array_equal(host(back.tensors[1], d["m"] * 8), o_aos.pool[: d["m"] * 8])


@pytest.mark.parametrize("pair", [("soa", 0, "aosoa", 32), ("aosoa", 32, "soa", 0), ("aosoa", 32, "aosoa", 128),
                                  ("aosoa", 128, "aosoa", 5)], ids=lambda p: "%s%d-%s%d" % p)
def test_field_major_to_field_major(pair):
    """SoA <-> AoSoA(B) and AoSoA(B) -> AoSoA(B') of a jagged collection:
    parents change layout, offsets and child values are copied."""
    sk, sb, dk, db = pair
    n = 3001
    s, o, d = tracks(n, seed=9, raw=True)
    o_aos = oracle.pack(o, d, "aos")
    o_src = oracle.convert(o, o_aos, sk, sb, m=d["m"])
    want = oracle.convert(o, o_src, dk, db, m=d["m"]).base
    nb = o.base_bytes(dk, db, n, d["m"])
    dst = dev_dest(s, dk, n, d["m"], db)
    mrn.convert(dev_view(s, o_src, o), dst)
    assert mrn.sync() == mrn.OK
    assert np.array_equal(host(dst.tensors[0], nb), want[:nb])


def test_aosoa_with_separate_offsets_and_child_columns():
    """A jagged AoSoA view may keep its offsets and child columns outside
    view.base; results equal the regions of the single-block form."""
    n, B = 2048 + 77, 32
    s, o, d = tracks(n, seed=21)
    m = d["m"]
    o_aos = oracle.pack(o, d, "aos")
    o_blk = oracle.convert(o, o_aos, "aosoa", B, m=m)
    blocks = garbage(s.required_bytes("aosoa", n, 0, B))
    offs = garbage((n + 1) * 4)
    kids = [garbage(m * 4) for _ in range(2)]
    dst = mrn.View(s, "aosoa", n, block=B, base=blocks, offsets=offs, child_columns=kids, m=m)
    mrn.convert(dev_view(s, o_aos, o), dst)
    assert mrn.sync() == mrn.OK
    nblk = oracle.region(o, o_blk, 0).size
    assert np.array_equal(host(blocks, nblk), oracle.region(o, o_blk, 0))
    assert np.array_equal(host(offs), oracle.region(o, o_blk, 1))
    for c in range(2):
        assert np.array_equal(host(kids[c]), oracle.region(o, o_blk, 2 + c))
    # and back to AoS from the split form
    back = dev_dest(s, "aos", n, m)
    mrn.convert(dst, back)
    assert mrn.sync() == mrn.OK
    assert np.array_equal(host(back.tensors[0], n * 24), o_aos.base[: n * 24])


def test_region_offsets_match_the_oracle():
    s, o = mrn.Schema(datagen.TRACKS), oracle.Schema(datagen.TRACKS)
    for n, m, B in [(0, 0, 32), (1, 3, 5), (1000, 20000, 128), (12345, 6789, 32)]:
        assert s.required_bytes("aosoa", n, m, B) == o.base_bytes("aosoa", B, n, m)
        for r in range(4):
            assert s.region_offset("aosoa", n, m, r, B) == o.fm_region_start("aosoa", B, n, m, r)


@pytest.mark.parametrize("n,osz,raw", [(300001, "u32", False), (262144, "u64", True)])
def test_large_soa_to_aos_parents_as_a_plain_conversion(n, osz, raw):
    """From 262,144 parents a SoA -> AoS conversion builds the parents as a
    plain conversion (their {length, begin} first as two columns): records
    and child pool equal the oracle's, u32 and u64 offsets, raw bits."""
    desc = [m if m[1] != "jagged" else (m[0], m[1], osz, m[3]) for m in datagen.TRACKS]
    s, o = mrn.Schema(desc), oracle.Schema(desc)
    d = datagen.workload("tracks", n, 17, raw=raw)
    o_aos = oracle.pack(o, d, "aos")
    o_soa = oracle.convert(o, o_aos, "soa", m=d["m"])
    src = mrn.View(s, "soa", n, base=dev(o_soa.base), m=d["m"])
    back = dev_dest(s, "aos", n, d["m"])
    mrn.convert(src, back)
    assert mrn.sync() == mrn.OK
    assert np.array_equal(host(back.tensors[0], n * o.stride), o_aos.base[: n * o.stride])
    assert np.array_equal(host(back.tensors[1], d["m"] * 8), o_aos.pool[: d["m"] * 8])
    # decreasing offsets are reported, not read past
    bad = o_soa.base.copy()
    st = o.soa_region_start(n, d["m"], s.ncols)
    osize = 4 if osz == "u32" else 8
    bad[st + 5 * osize: st + 6 * osize] = np.frombuffer(np.array([d["m"] + 10], "<u%d" % osize).tobytes(), np.uint8)
    mrn.convert(mrn.View(s, "soa", n, base=dev(bad), m=d["m"]), dev_dest(s, "aos", n, d["m"]))
    assert mrn.sync() == mrn.EINVAL


@pytest.mark.parametrize("case", ["canonical", "swapped_runs", "extra_records", "shuffled"])
def test_split_pool_checks(case, jagged_path):
    """A split run's check (the scan's, or the parents' local one) decides
    whether the pool can be converted as one plain conversion (pool record
    j -> child row j): only for a canonical pool that holds no other
    records.  Swapped runs, records beyond the children and a shuffled pool
    must take the fall-back pass; either way the offsets and child rows
    equal the oracle's, and child rows past the written count (capacity
    above the pool) keep their bytes."""
    n = 5 * 1024 + 333
    s, o, d = tracks(n, seed=61)
    o_aos = oracle.pack(o, d, "aos")
    m, lens = d["m"], d["lengths"]
    if case == "swapped_runs":
        order = np.arange(n)
        nz = [i for i in range(2048, 3072) if lens[i] > 0]
        order[nz[1]], order[nz[7]] = nz[7], nz[1]
        o_aos = oracle.shuffle_pool(o, o_aos, order, gap=0)
    elif case == "extra_records":  # canonical runs, then 50 records no parent owns
        pool = np.concatenate([o_aos.pool[: m * 8], np.full(50 * 8, 7, np.uint8)])
        o_aos = oracle.Side("aos", n, m + 50, base=o_aos.base, pool=pool)
    elif case == "shuffled":
        o_aos = oracle.shuffle_pool(o, o_aos, np.random.default_rng(5).permutation(n), gap=0)
    pool_n = o_aos.m
    cap = pool_n + 100
    o_soa = oracle.convert(o, o_aos, "soa", m=m)
    cols = [garbage(n * 4) for _ in range(3)]
    offs = garbage((n + 1) * 4)
    kids = [garbage(cap * 4) for _ in range(2)]
    dst = mrn.View(s, "soa", n, columns=cols, offsets=offs, child_columns=kids, m=cap)
    mrn.convert(dev_view(s, o_aos, o), dst)
    assert mrn.sync() == mrn.OK
    for c in range(3):
        assert np.array_equal(host(cols[c]), oracle.region(o, o_soa, c))
    assert np.array_equal(host(offs), oracle.region(o, o_soa, 3))
    for c in range(2):
        got = host(kids[c])
        assert np.array_equal(got[: m * 4], oracle.region(o, o_soa, 4 + c)), "child column %d" % c
        assert (got[m * 4:] == 0xA5).all(), "child rows past the count were written"
