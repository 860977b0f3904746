"""GPU parity of nested jagged members (children with a jagged member of
their own): AoS <-> single-block SoA and AoS <-> AoSoA(B) on canonical and
shuffled pools at both levels, sizes across many tiles, u32 and u64
offsets, and the errors each level reports, each equal to the oracle."""
import numpy as np
import pytest

import datagen
import oracle
import paper_2511_04853_b300 as mrn
from gpu_util import dev, garbage, host
from nested_util import shuffled_nested

pytestmark = pytest.mark.gpu
NESTED_SPLIT_DEFAULT = 1 << 18  # children from which level 0 of AoS -> field-major runs split (debug key 7)


@pytest.fixture(autouse=True, params=["level0_fused", "level0_split"])
def level0_path(request):
    """Every test of this module runs twice: level 0 of AoS -> field-major
    fused (its tiles gather the children and their descriptors), and split
    (the parents with the child pool's check, the pool as one staged
    conversion of the child record, the fused tiles again when the pool is
    not canonical)."""
    mrn.debug_set(7, -1 if request.param == "level0_fused" else 0)
    yield request.param
    mrn.debug_set(7, NESTED_SPLIT_DEFAULT)

SMALL = [
    [("a", "u8", 1), ("v", "jagged", "u32", [("x", "u16", 1), ("w", "jagged", "u32", [("y", "u8", 1)])])],
    [("v", "jagged", "u64", [("w", "jagged", "u32", [("y", "u64", 1), ("z", "u8", 3)]), ("x", "f32", 1)]),
     ("b", "u32", 2)],
    [("g", "group", [("p", "f64", 1), ("v", "jagged", "u32", [("x", "u8", 2),
                                                            ("w", "jagged", "u64", [("y", "u16", 1)])])])],
]


def fm_dest(s, kind, n, m, m2, block=0):
    return garbage(s.required_bytes_nested(kind, n, m, m2, block))


def to_fm(s, o, o_src, n, m, m2, kind, block):
    """Device AoS (from the oracle side) -> field-major; returns the bytes
    and the oracle's bytes of the same conversion."""
    want = oracle.convert(o, o_src, kind, block, m=m, m2=m2).base[: s.required_bytes_nested(kind, n, m, m2, block)]
    dst = fm_dest(s, kind, n, m, m2, block)
    src = mrn.View(s, "aos", n, base=dev(o_src.base), child_pool=dev(o_src.pool), m=o_src.m,
                   m2=o_src.m2, grandchild_pool=dev(o_src.gpool))
    mrn.convert(src, mrn.View(s, kind, n, block=block, base=dst, m=m, m2=m2))
    assert mrn.sync() == mrn.OK
    return host(dst, want.size), want, dst


def back_to_aos(s, o, dst, n, m, m2, kind, block):
    recs, pool, gpool = garbage(n * o.stride), garbage(m * o.child.stride), garbage(m2 * o.child.child.stride)
    mrn.convert(mrn.View(s, kind, n, block=block, base=dst, m=m, m2=m2),
                mrn.View(s, "aos", n, base=recs, child_pool=pool, m=m, m2=m2, grandchild_pool=gpool))
    assert mrn.sync() == mrn.OK
    return host(recs, n * o.stride), host(pool, m * o.child.stride), host(gpool, m2 * o.child.child.stride)


@pytest.mark.parametrize("n", [0, 1, 1000, 70001])
@pytest.mark.parametrize("kind,block", [("soa", 0), ("aosoa", 32), ("aosoa", 5)])
def test_tracks_nested_round_trip(n, kind, block):
    s, o = mrn.Schema(datagen.TRACKS_NESTED), oracle.Schema(datagen.TRACKS_NESTED)
    d = datagen.workload("tracks_nested", n, 3 + n % 7)
    aos = oracle.pack(o, d, "aos")
    m, m2 = d["m"], d["m2"]
    got, want, dst = to_fm(s, o, aos, n, m, m2, kind, block)
    assert np.array_equal(got, want)
    recs, pool, gpool = back_to_aos(s, o, dst, n, m, m2, kind, block)
    assert np.array_equal(recs, aos.base[: n * o.stride])
    assert np.array_equal(pool, aos.pool[: m * o.child.stride])
    assert np.array_equal(gpool, aos.gpool[: m2 * o.child.child.stride])


@pytest.mark.parametrize("k", range(len(SMALL)))
@pytest.mark.parametrize("n", [1, 7, 3001])
def test_shuffled_pools_raw_bits(k, n):
    desc = SMALL[k]
    s, o = mrn.Schema(desc), oracle.Schema(desc)
    d = datagen.jagged_random(desc, n, 50 + n + k, mean_len=3.0, max_len=8)
    aos = oracle.pack(o, d, "aos")
    recs, pool, gpool, mp, m2p = shuffled_nested(o, aos, seed=k * 100 + n)
    src_o = oracle.Side("aos", n, mp, base=recs, pool=pool, gpool=gpool, m2=m2p)
    m, m2 = d["m"], d["m2"]
    for kind, block in (("soa", 0), ("aosoa", 32)):
        got, want, _ = to_fm(s, o, src_o, n, m, m2, kind, block)
        assert np.array_equal(got, want), (kind, block)


def test_capacity_and_bad_indices_are_reported():
    s, o = mrn.Schema(datagen.TRACKS_NESTED), oracle.Schema(datagen.TRACKS_NESTED)
    n = 5000
    d = datagen.workload("tracks_nested", n, 11)
    aos = oracle.pack(o, d, "aos")
    m, m2 = d["m"], d["m2"]
    src = mrn.View(s, "aos", n, base=dev(aos.base), child_pool=dev(aos.pool), m=m, m2=m2,
                   grandchild_pool=dev(aos.gpool))
    # too few children slots: recorded by the first level (the children's
    # count never returns to the host), reported at the next sync
    small = fm_dest(s, "soa", n, m - 1, m2)
    assert mrn.convert_status(src, mrn.View(s, "soa", n, base=small, m=m - 1, m2=m2)) == mrn.OK
    assert mrn.sync() == mrn.ESIZE
    # too few grandchild slots: recorded by the second level
    dst = fm_dest(s, "soa", n, m, m2 - 1)
    assert mrn.convert_status(src, mrn.View(s, "soa", n, base=dst, m=m, m2=m2 - 1)) == mrn.OK
    assert mrn.sync() == mrn.ESIZE
    # a child whose samples run past the grandchild pool
    pool = aos.pool.copy()
    pool[o.child.begin_off: o.child.begin_off + 8] = np.array([m2], "<u8").view(np.uint8)
    pool[o.child.len_off: o.child.len_off + 4] = np.array([1], "<u4").view(np.uint8)
    bad = mrn.View(s, "aos", n, base=dev(aos.base), child_pool=dev(pool), m=m, m2=m2,
                   grandchild_pool=dev(aos.gpool))
    dst = fm_dest(s, "soa", n, m, m2 + 1)
    assert mrn.convert_status(bad, mrn.View(s, "soa", n, base=dst, m=m, m2=m2 + 1)) == mrn.OK
    assert mrn.sync() == mrn.EINVAL
    # afterwards a good conversion runs normally
    got, want, _ = to_fm(s, o, aos, n, m, m2, "soa", 0)
    assert np.array_equal(got, want)


def test_other_paths_refuse_nested_members():
    import torch
    s = mrn.Schema(datagen.TRACKS_NESTED)
    n, m, m2 = 10, 20, 30
    a = fm_dest(s, "soa", n, m, m2)
    b = fm_dest(s, "aosoa", n, m, m2, 32)
    src = mrn.View(s, "soa", n, base=a, m=m, m2=m2)
    assert mrn.convert_status(src, mrn.View(s, "aosoa", n, block=32, base=b, m=m, m2=m2)) == mrn.EUNSUPPORTED
    recs, pool, gpool = garbage(n * s.stride), garbage(m * 24), garbage(m2 * 4)
    aos = mrn.View(s, "aos", n, base=recs, child_pool=pool, m=m, m2=m2, grandchild_pool=gpool)
    with pytest.raises(mrn.MrnError):
        mrn.Batch([(aos, mrn.View(s, "soa", n, base=a, m=m, m2=m2))], use_graph=False)
    h = torch.zeros(n * s.stride, dtype=torch.uint8).pin_memory()
    hv = mrn.View(s, "aos", n, base=h, child_pool=h, m=m, m2=m2, grandchild_pool=h, mem="pinned")
    st = mrn.lib().mrn_transfer_convert(hv.ref, mrn.View(s, "soa", n, base=a, m=m, m2=m2).ref, None,
                                        mrn.mrn._stream(None))
    assert st == mrn.EUNSUPPORTED


def test_scratch_is_kept_between_calls_and_released():
    """A 2,097,152-parent nested conversion holds about 0.5 GB of scratch (a
    length and a begin per child): the library's pool keeps it reserved
    after the call, so that the next call does not map it again, and
    mrn_scratch_release returns it to the device.  Results are unchanged
    throughout: equal outputs before and after the release, and the round
    trip gives back the source's bytes (canonical pools, 20 hits per track
    and 3 samples per hit)."""
    import torch
    s = mrn.Schema(datagen.TRACKS_NESTED)
    n, per, per2 = 1 << 21, 20, 3
    m, m2 = n * per, n * per * per2
    g = torch.Generator(device="cuda")
    g.manual_seed(11)

    def records(count, stride, length, len_off, beg_off):
        r = torch.randint(0, 256, (count * stride,), dtype=torch.uint8, device="cuda", generator=g)
        rv = r.view(count, stride)
        lens = torch.full((count,), length, dtype=torch.int32, device="cuda")
        rv[:, len_off:len_off + 4].copy_(lens.view(torch.uint8).view(count, 4))
        rv[:, len_off + 4:beg_off].zero_()
        begs = torch.arange(count, dtype=torch.int64, device="cuda") * length
        rv[:, beg_off:beg_off + 8].copy_(begs.view(torch.uint8).view(count, 8))
        return r
    recs, pool = records(n, 24, per, 12, 16), records(m, 24, per2, 8, 16)
    gpool = torch.randint(0, 256, (m2 * 4,), dtype=torch.uint8, device="cuda", generator=g)
    fm = torch.empty(s.required_bytes_nested("soa", n, m, m2), dtype=torch.uint8, device="cuda")
    a = mrn.View(s, "aos", n, base=recs, child_pool=pool, m=m, m2=m2, grandchild_pool=gpool)
    f = mrn.View(s, "soa", n, base=fm, m=m, m2=m2)
    device = torch.cuda.current_device()
    mrn.scratch_release(device)
    mrn.convert(a, f)
    assert mrn.sync() == mrn.OK
    first = fm.clone()
    torch.cuda.synchronize()
    kept = torch.cuda.mem_get_info()[0]
    mrn.scratch_release(device)
    freed = torch.cuda.mem_get_info()[0] - kept
    assert freed >= 400 << 20, freed
    fm.fill_(0)
    mrn.convert(a, f)
    assert mrn.sync() == mrn.OK
    assert torch.equal(fm, first)
    recs2, pool2, gpool2 = torch.empty_like(recs), torch.empty_like(pool), torch.empty_like(gpool)
    mrn.convert(f, mrn.View(s, "aos", n, base=recs2, child_pool=pool2, m=m, m2=m2, grandchild_pool=gpool2))
    assert mrn.sync() == mrn.OK
    assert torch.equal(recs2, recs) and torch.equal(pool2, pool) and torch.equal(gpool2, gpool)
    mrn.scratch_release(device)
