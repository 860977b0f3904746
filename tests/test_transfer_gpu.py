"""GPU parity of transfer-and-convert between host and device views (the
chunked copy/convert pipeline): every chunk size, direction and layout pair
must give the oracle's bytes."""
import numpy as np
import pytest

import datagen
import oracle
import paper_2511_04853_b300 as mrn
from gpu_util import dev, garbage, host, torch

pytestmark = pytest.mark.gpu


def pinned(nbytes, fill=0xA5):
    return torch().full((max(1, int(nbytes)),), fill, dtype=torch().uint8).pin_memory()


def host_side(arr, pin=True):
    a = np.ascontiguousarray(arr).view(np.uint8).reshape(-1)
    if a.size == 0:
        a = np.zeros(1, np.uint8)
    t = torch().from_numpy(a.copy())
    return t.pin_memory() if pin else t


def cells(n, seed=1):
    return mrn.Schema(datagen.CELLS), oracle.Schema(datagen.CELLS), datagen.workload("cells", n, seed)


@pytest.mark.parametrize("chunk", [64 << 10, 1 << 20, 16 << 20])
@pytest.mark.parametrize("n", [1, 200000, 70001])
def test_h2d_aos_to_soa_chunk_sweep(chunk, n):
    s, o, d = cells(n)
    o_aos = oracle.pack(o, d, "aos")
    o_soa = oracle.convert(o, o_aos, "soa")
    dst = garbage(s.required_bytes("soa", n))
    mrn.transfer_convert(mrn.View(s, "aos", n, base=host_side(o_aos.base), mem="pinned"),
                         mrn.View(s, "soa", n, base=dst), chunk_bytes=chunk, n_slots=4)
    assert mrn.sync() == mrn.OK
    assert np.array_equal(host(dst, o_soa.base.size), o_soa.base)


@pytest.mark.parametrize("pair", [("soa", 0, "aos", 0), ("aosoa", 32, "aos", 0), ("aos", 0, "aosoa", 32),
                                  ("aos", 0, "soa", 0), ("soa", 0, "aosoa", 128)])
@pytest.mark.parametrize("chunk", [256 << 10, 4 << 20])
def test_d2h_layout_pairs(pair, chunk):
    sk, sb, dk, db = pair
    n = 100003
    s, o, d = cells(n, seed=3)
    o_src = oracle.pack(o, d, sk, sb)
    o_dst = oracle.convert(o, o_src, dk, db)
    hdst = pinned(o.base_bytes(dk, db, n))
    mrn.transfer_convert(mrn.View(s, sk, n, block=sb, base=dev(o_src.base)),
                         mrn.View(s, dk, n, block=db, base=hdst, mem="pinned"), chunk_bytes=chunk)
    assert mrn.sync() == mrn.OK
    assert np.array_equal(hdst.numpy()[: o_dst.base.size], o_dst.base)


@pytest.mark.parametrize("pair", [("aosoa", 32, "soa", 0), ("soa", 0, "aosoa", 32), ("aosoa", 128, "aos", 0)])
def test_h2d_layout_pairs(pair):
    sk, sb, dk, db = pair
    n = 50001
    s, o, d = cells(n, seed=4)
    o_src = oracle.pack(o, d, sk, sb)
    o_dst = oracle.convert(o, o_src, dk, db)
    dst = garbage(s.required_bytes(dk, n, 0, db))
    mrn.transfer_convert(mrn.View(s, sk, n, block=sb, base=host_side(o_src.base), mem="pinned"),
                         mrn.View(s, dk, n, block=db, base=dst), chunk_bytes=1 << 20)
    assert mrn.sync() == mrn.OK
    assert np.array_equal(host(dst, o_dst.base.size), o_dst.base)


def test_points_gaps_and_pageable_memory():
    """10,000 points to a single-block SoA whose columns have alignment
    holes, from pageable host memory, and back into pageable memory."""
    n = 10000
    s, o = mrn.Schema(datagen.POINTS), oracle.Schema(datagen.POINTS)
    d = datagen.workload("points", n, 0)
    o_aos = oracle.pack(o, d, "aos")
    o_soa = oracle.convert(o, o_aos, "soa")
    dst = garbage(s.required_bytes("soa", n))
    mrn.transfer_convert(mrn.View(s, "aos", n, base=host_side(o_aos.base, pin=False), mem="host"),
                         mrn.View(s, "soa", n, base=dst), chunk_bytes=32 << 10)
    assert mrn.sync() == mrn.OK
    assert np.array_equal(host(dst, o_soa.base.size), o_soa.base)
    back = np.full(o_soa.base.size, 0xA5, np.uint8)
    mrn.transfer_convert(mrn.View(s, "aos", n, base=dev(o_aos.base)),
                         mrn.View(s, "soa", n, base=back, mem="host"), chunk_bytes=64 << 10)
    assert mrn.sync() == mrn.OK
    assert np.array_equal(back, o_soa.base)


def test_same_layout_is_a_copy():
    n = 12345
    s, o, d = cells(n)
    o_aos = oracle.pack(o, d, "aos")
    dst = garbage(n * 24)
    mrn.transfer_convert(mrn.View(s, "aos", n, base=host_side(o_aos.base), mem="pinned"),
                         mrn.View(s, "aos", n, base=dst))
    assert mrn.sync() == mrn.OK
    assert np.array_equal(host(dst, n * 24), o_aos.base)


def test_jagged_both_directions():
    n = 30000
    s, o = mrn.Schema(datagen.TRACKS), oracle.Schema(datagen.TRACKS)
    d = datagen.workload("tracks", n, 2)
    o_aos = oracle.pack(o, d, "aos")
    o_soa = oracle.convert(o, o_aos, "soa", m=d["m"])
    dst = garbage(s.required_bytes("soa", n, d["m"]))
    mrn.transfer_convert(mrn.View(s, "aos", n, base=host_side(o_aos.base), child_pool=host_side(o_aos.pool),
                                  m=d["m"], mem="pinned"),
                         mrn.View(s, "soa", n, base=dst, m=d["m"]))
    assert mrn.sync() == mrn.OK
    assert np.array_equal(host(dst, o_soa.base.size), o_soa.base)
    hb, hp = pinned(n * 24), pinned(d["m"] * 8)
    mrn.transfer_convert(mrn.View(s, "soa", n, base=dst, m=d["m"]),
                         mrn.View(s, "aos", n, base=hb, child_pool=hp, m=d["m"], mem="pinned"))
    assert mrn.sync() == mrn.OK
    assert np.array_equal(hb.numpy()[: n * 24], o_aos.base[: n * 24])
    assert np.array_equal(hp.numpy()[: d["m"] * 8], o_aos.pool[: d["m"] * 8])


def test_host_to_host_rejected():
    s = mrn.Schema(datagen.CELLS)
    a = np.zeros(240, np.uint8)
    st = mrn.lib().mrn_transfer_convert(mrn.View(s, "aos", 10, base=a, mem="host").ref,
                                        mrn.View(s, "soa", 10, base=a, mem="host").ref, None, None)
    assert st == mrn.EINVAL


def test_both_directions_on_several_streams():
    """Host -> device and device -> host transfers issued on four streams
    (they overlap on the two direction pipelines) give the oracle's bytes,
    and the round trip host AoS -> device SoA -> AoSoA(32) -> host AoS
    reproduces every collection."""
    t = torch()
    s, o = mrn.Schema(datagen.CELLS), oracle.Schema(datagen.CELLS)
    streams = [t.cuda.Stream() for _ in range(4)]
    jobs = []
    for i in range(8):
        n = 50000 + 977 * i
        d = datagen.workload("cells", n, 40 + i)
        o_aos = oracle.pack(o, d, "aos")
        jobs.append((n, o_aos, host_side(o_aos.base), garbage(s.required_bytes("soa", n)),
                     garbage(s.required_bytes("aosoa", n, 0, 32)), pinned(n * 24)))
    t.cuda.synchronize()
    for i, (n, o_aos, h_in, d_soa, d_blk, h_out) in enumerate(jobs):
        st = streams[i % 4]
        soa = mrn.View(s, "soa", n, base=d_soa)
        blk = mrn.View(s, "aosoa", n, block=32, base=d_blk)
        mrn.transfer_convert(mrn.View(s, "aos", n, base=h_in, mem="pinned"), soa, chunk_bytes=256 << 10,
                             n_slots=4, stream=st)
        mrn.convert(soa, blk, stream=st)
        mrn.transfer_convert(blk, mrn.View(s, "aos", n, base=h_out, mem="pinned"), chunk_bytes=256 << 10,
                             n_slots=4, stream=st)
    t.cuda.synchronize()
    assert mrn.sync() == mrn.OK
    for n, o_aos, h_in, d_soa, d_blk, h_out in jobs:
        want_soa = oracle.convert(o, o_aos, "soa").base
        assert np.array_equal(host(d_soa, want_soa.size), want_soa)
        assert np.array_equal(h_out.numpy()[: n * 24], o_aos.base[: n * 24])


@pytest.mark.parametrize("pair", [(("aos", 0), ("soa", 0)), (("aos", 0), ("aosoa", 32)), (("soa", 0), ("aos", 0)),
                                  (("aosoa", 128), ("soa", 0))], ids=lambda p: "%s%d-%s%d" % (p[0] + p[1]))
@pytest.mark.parametrize("name,n", [("cells", 70001), ("points", 10000), ("sensor", 999)])
def test_zero_copy_both_directions(pair, name, n):
    """Zero-copy transfer-and-convert: the kernel reads (host -> device) or
    writes (device -> host) the pinned host buffer directly; bytes equal the
    oracle's, alignment holes and AoSoA tail slots included."""
    (sk, sb), (dk, db) = pair
    desc = datagen.WORKLOAD_SCHEMAS.get(name) or getattr(datagen, name.upper())
    s, o = mrn.Schema(desc), oracle.Schema(desc)
    if name in datagen.WORKLOAD_SCHEMAS:
        d = datagen.workload(name, n, 31)
    else:
        d = datagen.random_columns(desc, n, 31)
    o_src = oracle.pack(o, d, sk, sb)
    want = oracle.convert(o, o_src, dk, db).base
    nb = s.required_bytes(dk, n, 0, db)
    # host -> device
    dst = garbage(nb)
    mrn.transfer_convert(mrn.View(s, sk, n, block=sb, base=host_side(o_src.base), mem="pinned"),
                         mrn.View(s, dk, n, block=db, base=dst), zero_copy=True)
    assert mrn.sync() == mrn.OK
    assert np.array_equal(host(dst, want.size), want)
    # device -> host
    h = pinned(nb)
    mrn.transfer_convert(mrn.View(s, sk, n, block=sb, base=dev(o_src.base)),
                         mrn.View(s, dk, n, block=db, base=h, mem="pinned"), zero_copy=True)
    torch().cuda.synchronize()
    assert mrn.sync() == mrn.OK
    assert np.array_equal(h.numpy()[: want.size], want)


def test_zero_copy_rejections():
    s = mrn.Schema(datagen.TRACKS)
    buf = garbage(1 << 12)
    hp = pinned(1 << 12)
    src = mrn.View(s, "aos", 10, base=hp, child_pool=hp, m=1, mem="pinned")
    assert lib_status(src, mrn.View(s, "soa", 10, base=buf, m=1)) == mrn.EUNSUPPORTED
    c = mrn.Schema(datagen.CELLS)
    pageable = torch().zeros(1 << 12, dtype=torch().uint8)
    assert lib_status(mrn.View(c, "aos", 10, base=pageable, mem="host"),
                      mrn.View(c, "soa", 10, base=buf)) == mrn.EINVAL


def lib_status(src, dst):
    import ctypes
    from paper_2511_04853_b300 import mrn as binding
    opts = binding.TransferOpts(0, 0, binding.TRANSFER_ZERO_COPY)
    return binding.lib().mrn_transfer_convert(src.ref, dst.ref, ctypes.byref(opts), None)


@pytest.mark.parametrize("B", [32, 128])
def test_jagged_aosoa_both_directions(B):
    """Host AoS -> device jagged AoSoA(B) and device AoSoA(B) -> host AoS
    through the transfer engine (host single-block holes zeroed)."""
    s, o = mrn.Schema(datagen.TRACKS), oracle.Schema(datagen.TRACKS)
    n = 7777
    d = datagen.workload("tracks", n, 61)
    m = d["m"]
    o_aos = oracle.pack(o, d, "aos")
    o_blk = oracle.convert(o, o_aos, "aosoa", B, m=m)
    nb = o.base_bytes("aosoa", B, n, m)
    dst = garbage(nb)
    src = mrn.View(s, "aos", n, base=host_side(o_aos.base), child_pool=host_side(o_aos.pool), m=m, mem="pinned")
    mrn.transfer_convert(src, mrn.View(s, "aosoa", n, block=B, base=dst, m=m))
    assert mrn.sync() == mrn.OK
    assert np.array_equal(host(dst, nb), o_blk.base[:nb])
    h_rec, h_pool = pinned(n * 24), pinned(m * 8)
    mrn.transfer_convert(mrn.View(s, "aosoa", n, block=B, base=dev(o_blk.base), m=m),
                         mrn.View(s, "aos", n, base=h_rec, child_pool=h_pool, m=m, mem="pinned"))
    torch().cuda.synchronize()
    assert mrn.sync() == mrn.OK
    assert np.array_equal(h_rec.numpy()[: n * 24], o_aos.base[: n * 24])
    assert np.array_equal(h_pool.numpy()[: m * 8], o_aos.pool[: m * 8])


def test_back_to_back_calls_on_different_streams_share_staging_safely():
    """Host -> device calls issued on two streams with no synchronisation
    between them use the same staging memory: a chunked call on stream A
    followed by a jagged (whole-source) call on stream B, then a chunked
    call with another chunk size on stream A.  Each result equals the
    oracle's."""
    t = torch()
    a, b = t.cuda.Stream(), t.cuda.Stream()
    n = 200000
    s, o, d = cells(n, seed=11)
    o_aos = oracle.pack(o, d, "aos")
    o_soa = oracle.convert(o, o_aos, "soa")
    st, ot = mrn.Schema(datagen.TRACKS), oracle.Schema(datagen.TRACKS)
    nt = 30000
    dt = datagen.workload("tracks", nt, 12)
    ot_aos = oracle.pack(ot, dt, "aos")
    ot_soa = oracle.convert(ot, ot_aos, "soa")
    h_cells = host_side(o_aos.base)
    h_rec, h_pool = host_side(ot_aos.base), host_side(ot_aos.pool)
    d1, d3 = garbage(s.required_bytes("soa", n)), garbage(s.required_bytes("soa", n))
    d2 = garbage(st.required_bytes("soa", nt, dt["m"]))
    t.cuda.synchronize()
    mrn.transfer_convert(mrn.View(s, "aos", n, base=h_cells, mem="pinned"), mrn.View(s, "soa", n, base=d1),
                         chunk_bytes=256 << 10, n_slots=2, stream=a)
    mrn.transfer_convert(mrn.View(st, "aos", nt, base=h_rec, child_pool=h_pool, m=dt["m"], mem="pinned"),
                         mrn.View(st, "soa", nt, base=d2, m=dt["m"]), stream=b)
    mrn.transfer_convert(mrn.View(s, "aos", n, base=h_cells, mem="pinned"), mrn.View(s, "soa", n, base=d3),
                         chunk_bytes=1 << 20, n_slots=3, stream=a)
    t.cuda.synchronize()
    assert mrn.sync() == mrn.OK
    assert np.array_equal(host(d1, o_soa.base.size), o_soa.base)
    assert np.array_equal(host(d2, ot_soa.base.size), ot_soa.base)
    assert np.array_equal(host(d3, o_soa.base.size), o_soa.base)


def test_pipelined_calls_mixed_schemas_whole_sources_and_write_order():
    """Host -> device calls on two streams with no synchronisation between
    them: chunked calls of two schemas with the same chunk size (they share
    the staging slots, each waiting only for the slots it reuses), three
    jagged calls in a row (whole-source buffers taken in turn) and, last,
    an equal-layout copy into a destination an earlier call converted into
    (destinations are written in call order).  Every result equals the
    oracle's."""
    t = torch()
    streams = [t.cuda.Stream(), t.cuda.Stream()]
    n_c, n_p = 150000, 90001
    sc, oc, dc = cells(n_c, seed=21)
    c_soa = oracle.convert(oc, oracle.pack(oc, dc, "aos"), "soa")
    h_c = host_side(oracle.pack(oc, dc, "aos").base)
    c2_soa = oracle.convert(oc, oracle.pack(oc, datagen.workload("cells", n_c, 23), "aos"), "soa")
    h_c2 = host_side(c2_soa.base)
    sp, op = mrn.Schema(datagen.POINTS), oracle.Schema(datagen.POINTS)
    p_aos = oracle.pack(op, datagen.workload("points", n_p, 22), "aos")
    p_soa = oracle.convert(op, p_aos, "soa")
    h_p = host_side(p_aos.base)
    st, ot = mrn.Schema(datagen.TRACKS), oracle.Schema(datagen.TRACKS)
    tracks = []
    for k, nt in enumerate((20000, 35001, 12345)):
        dt = datagen.workload("tracks", nt, 30 + k)
        a = oracle.pack(ot, dt, "aos")
        tracks.append((nt, dt["m"], host_side(a.base), host_side(a.pool), oracle.convert(ot, a, "soa")))
    d_c1, d_c2 = garbage(sc.required_bytes("soa", n_c)), garbage(sc.required_bytes("soa", n_c))
    d_p1, d_p2 = garbage(sp.required_bytes("soa", n_p)), garbage(sp.required_bytes("soa", n_p))
    d_t = [garbage(st.required_bytes("soa", nt, m)) for nt, m, _, _, _ in tracks]
    calls = [
        (mrn.View(sc, "aos", n_c, base=h_c, mem="pinned"), mrn.View(sc, "soa", n_c, base=d_c1)),
        (mrn.View(sp, "aos", n_p, base=h_p, mem="pinned"), mrn.View(sp, "soa", n_p, base=d_p1)),
        (mrn.View(st, "aos", tracks[0][0], base=tracks[0][2], child_pool=tracks[0][3], m=tracks[0][1], mem="pinned"),
         mrn.View(st, "soa", tracks[0][0], base=d_t[0], m=tracks[0][1])),
        (mrn.View(sc, "aos", n_c, base=h_c, mem="pinned"), mrn.View(sc, "soa", n_c, base=d_c2)),
        (mrn.View(st, "aos", tracks[1][0], base=tracks[1][2], child_pool=tracks[1][3], m=tracks[1][1], mem="pinned"),
         mrn.View(st, "soa", tracks[1][0], base=d_t[1], m=tracks[1][1])),
        (mrn.View(st, "aos", tracks[2][0], base=tracks[2][2], child_pool=tracks[2][3], m=tracks[2][1], mem="pinned"),
         mrn.View(st, "soa", tracks[2][0], base=d_t[2], m=tracks[2][1])),
        (mrn.View(sp, "aos", n_p, base=h_p, mem="pinned"), mrn.View(sp, "soa", n_p, base=d_p2)),
        (mrn.View(sc, "soa", n_c, base=h_c2, mem="pinned"), mrn.View(sc, "soa", n_c, base=d_c1)),
    ]
    t.cuda.synchronize()
    for i, (src, dst) in enumerate(calls):
        mrn.transfer_convert(src, dst, chunk_bytes=256 << 10, n_slots=3, stream=streams[i % 2])
    t.cuda.synchronize()
    assert mrn.sync() == mrn.OK
    assert np.array_equal(host(d_c1, c2_soa.base.size), c2_soa.base), "equal-layout copy not last"
    assert np.array_equal(host(d_c2, c_soa.base.size), c_soa.base)
    assert np.array_equal(host(d_p1, p_soa.base.size), p_soa.base)
    assert np.array_equal(host(d_p2, p_soa.base.size), p_soa.base)
    for k, (nt, m, _, _, want) in enumerate(tracks):
        assert np.array_equal(host(d_t[k], want.base.size), want.base), "tracks call %d" % k
