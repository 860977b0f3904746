"""GPU parity of the batched form: many collections of mixed schemas, sizes
and layout pairs in one persistent launch (with and without a CUDA graph)
must each equal the oracle, and equal the one-launch-per-collection result;
graph replays after the inputs change, job-table updates and the autotuner
must keep the results exact."""
import numpy as np
import pytest

import datagen
import oracle
import paper_2511_04853_b300 as mrn
from gpu_util import dev, dev_dest, garbage, host

pytestmark = pytest.mark.gpu

NAMES = ["points", "cells", "tracks"]
KINDS = [("aos", 0), ("soa", 0), ("aosoa", 32), ("aosoa", 128), ("aosoa", 5)]


def make_jobs(seed, count, max_n=20000):
    rng = np.random.default_rng(seed)
    jobs = []
    for j in range(count):
        name = NAMES[rng.integers(0, 3)]
        n = int(round(10 ** rng.uniform(0, np.log10(max_n))))
        desc = datagen.WORKLOAD_SCHEMAS[name]
        s, o = mrn.Schema(desc), oracle.Schema(desc)
        d = datagen.workload(name, n, seed * 1000 + j)
        if name == "tracks":
            o_aos = oracle.pack(o, d, "aos")
            o_soa = oracle.convert(o, o_aos, "soa", m=d["m"])
            if rng.integers(0, 2) == 0:
                src = mrn.View(s, "aos", n, base=dev(o_aos.base), child_pool=dev(o_aos.pool), m=d["m"])
                dst = dev_dest(s, "soa", n, d["m"])
                want = o_soa.base
            else:
                src = mrn.View(s, "soa", n, base=dev(o_soa.base), m=d["m"])
                dst = dev_dest(s, "aos", n, d["m"])
                want = np.concatenate([o_aos.base[: n * 24], o_aos.pool[: d["m"] * 8]])
        else:
            sk, sb = KINDS[rng.integers(0, len(KINDS))]
            dk, db = KINDS[rng.integers(0, len(KINDS))]
            if (sk, sb) == (dk, db) or (sk == dk == "aos"):
                sk, sb, dk, db = "aos", 0, "soa", 0
            o_src = oracle.pack(o, d, sk, sb)
            o_dst = oracle.convert(o, o_src, dk, db)
            src = mrn.View(s, sk, n, block=sb, base=dev(o_src.base))
            dst = dev_dest(s, dk, n, 0, db)
            want = o_dst.base
        jobs.append((src, dst, want, name))
    return jobs


def result(dst, want, name):
    if name == "tracks" and dst.tensors[1] is not None:
        n = dst.s.n_records
        return np.concatenate([host(dst.tensors[0], n * 24), host(dst.tensors[1], dst.s.n_children * 8)])
    return host(dst.tensors[0], want.size)


@pytest.mark.parametrize("use_graph", [True, False])
def test_mixed_batch_matches_oracle(use_graph):
    jobs = make_jobs(7, 60)
    b = mrn.Batch([(s, d) for s, d, _, _ in jobs], use_graph=use_graph)
    b.launch()
    assert mrn.sync() == mrn.OK
    for i, (s, d, want, name) in enumerate(jobs):
        assert np.array_equal(result(d, want, name), want), "job %d (%s)" % (i, name)
    # the per-collection baseline gives the same bytes
    for _, d, _, _ in jobs:
        d.tensors[0].fill_(0xA5)
    b.launch_per_job()
    assert mrn.sync() == mrn.OK
    for i, (s, d, want, name) in enumerate(jobs):
        assert np.array_equal(result(d, want, name), want), "per-job %d" % i


def test_graph_replay_sees_new_inputs():
    n = 30000
    s, o = mrn.Schema(datagen.CELLS), oracle.Schema(datagen.CELLS)
    src_t = garbage(n * 24)
    dst = dev_dest(s, "aosoa", n, 0, 32)
    b = mrn.Batch([(mrn.View(s, "aos", n, base=src_t), dst)], use_graph=True)
    for seed in (1, 2, 3):
        d = datagen.workload("cells", n, seed)
        o_aos = oracle.pack(o, d, "aos")
        src_t.copy_(dev(o_aos.base))
        b.launch()
        assert mrn.sync() == mrn.OK
        want = oracle.convert(o, o_aos, "aosoa", 32).base
        assert np.array_equal(host(dst.tensors[0], want.size), want)


def test_update_repoints_a_job():
    n = 5000
    s, o = mrn.Schema(datagen.POINTS), oracle.Schema(datagen.POINTS)
    d1, d2 = datagen.workload("points", n, 1), datagen.workload("points", n, 2)
    a1, a2 = oracle.pack(o, d1, "aos"), oracle.pack(o, d2, "aos")
    dst1, dst2 = dev_dest(s, "soa", n), dev_dest(s, "soa", n)
    b = mrn.Batch([(mrn.View(s, "aos", n, base=dev(a1.base)), dst1)], use_graph=True)
    b.update(0, mrn.View(s, "aos", n, base=dev(a2.base)), dst2)
    b.launch()
    assert mrn.sync() == mrn.OK
    want = oracle.convert(o, a2, "soa").base
    assert np.array_equal(host(dst2.tensors[0], want.size), want)


def test_autotune_then_convert_still_exact():
    s, o = mrn.Schema(datagen.CELLS), oracle.Schema(datagen.CELLS)
    r = mrn.autotune(s, "aos", "soa", 1 << 20)
    assert r["gbps"] > 0 and r["tile_records"] % 32 == 0 and r["threads"] in (128, 256)
    n = 200000
    d = datagen.workload("cells", n, 1)
    o_aos = oracle.pack(o, d, "aos")
    dst = dev_dest(s, "soa", n)
    mrn.convert(mrn.View(s, "aos", n, base=dev(o_aos.base)), dst)
    assert mrn.sync() == mrn.OK
    want = oracle.convert(o, o_aos, "soa").base
    assert np.array_equal(host(dst.tensors[0], want.size), want)
    mrn.autotune_clear()


@pytest.fixture(params=["split", "fused"])
def jagged_path(request):
    """Batches split their jagged AoS jobs by default: the parents (whose
    job also checks, record by record, that the pool is canonical) in the
    first persistent launch, the pool in the second (skipped unless
    canonical), and a fall-back pass that converts the jobs whose pools
    are not canonical whole again; debug key 4 < 0 keeps them fused."""
    if request.param == "fused":
        mrn.debug_set(4, -1)
    yield request.param
    mrn.debug_set(4, 2**63 - 1)


def test_jagged_jobs_shuffled_pools_many_tiles(jagged_path):
    """Jagged jobs of many tiles (look-back across CTAs), canonical and
    shuffled child pools (with and without records beyond the children),
    between plain conversions, in one launch."""
    pairs, checks = [], []
    for j, n in enumerate([3000, 41000, 257, 25000, 60000]):
        s, o = mrn.Schema(datagen.TRACKS), oracle.Schema(datagen.TRACKS)
        d = datagen.workload("tracks", n, 500 + j)
        o_aos = oracle.pack(o, d, "aos")
        if j % 2:
            order = np.random.default_rng(j).permutation(n)
            o_aos = oracle.shuffle_pool(o, o_aos, order, gap=1 if j == 1 else 0)
        want = oracle.convert(o, o_aos, "soa", m=d["m"]).base
        src = mrn.View(s, "aos", n, base=dev(o_aos.base), child_pool=dev(o_aos.pool), m=o_aos.m)
        dst = dev_dest(s, "soa", n, d["m"])
        pairs.append((src, dst))
        checks.append((dst, want))
        c_s, c_o = mrn.Schema(datagen.CELLS), oracle.Schema(datagen.CELLS)
        cd = datagen.workload("cells", 5000 + j, 600 + j)
        c_src = oracle.pack(c_o, cd, "aos")
        c_dst = dev_dest(c_s, "aosoa", 5000 + j, 0, 32)
        pairs.append((mrn.View(c_s, "aos", 5000 + j, base=dev(c_src.base)), c_dst))
        checks.append((c_dst, oracle.convert(c_o, c_src, "aosoa", 32).base))
    b = mrn.Batch(pairs, use_graph=True)
    for _ in range(2):
        for dst, _ in checks:
            dst.tensors[0].fill_(0xA5)
        b.launch()
        assert mrn.sync() == mrn.OK
        for k, (dst, want) in enumerate(checks):
            assert np.array_equal(host(dst.tensors[0], want.size), want), "job %d" % k


def test_batch_lookback_wait_is_bounded(jagged_path):
    """Host-side fault injection: jagged tile 1 of a batched job never
    publishes its sum, so the later look-backs must expire (1 ms bound) and
    report MRN_ETIMEOUT; batches built afterwards run normally.  A split
    job's look-back is its fall-back pass's, so its pool is shuffled (not
    canonical) to make that pass run."""
    n = 4 * 8192  # at least four tiles of up to 1,024 parents
    s, o = mrn.Schema(datagen.TRACKS), oracle.Schema(datagen.TRACKS)
    d = datagen.workload("tracks", n, 3)
    o_aos = oracle.pack(o, d, "aos")
    if jagged_path == "split":
        o_aos = oracle.shuffle_pool(o, o_aos, np.random.default_rng(2).permutation(n), gap=0)
    src = mrn.View(s, "aos", n, base=dev(o_aos.base), child_pool=dev(o_aos.pool), m=d["m"])
    try:
        mrn.debug_set(2, 1_000_000)
        mrn.debug_set(1, 1)
        b = mrn.Batch([(src, dev_dest(s, "soa", n, d["m"]))], use_graph=False)
    finally:
        mrn.debug_set(1, -1)
        mrn.debug_set(2, 2_000_000_000)
    b.launch()
    assert mrn.sync() == mrn.ETIMEOUT
    dst = dev_dest(s, "soa", n, d["m"])
    b2 = mrn.Batch([(src, dst)], use_graph=False)
    b2.launch()
    assert mrn.sync() == mrn.OK
    want = oracle.convert(o, o_aos, "soa", m=d["m"]).base
    assert np.array_equal(host(dst.tensors[0], want.size), want)


def test_partial_tiles_in_one_batch():
    """Collections whose sizes cut the staged tiles at every kind of place,
    all in one launch (staged partial tiles and direct remainders side by
    side with full tiles)."""
    pairs, checks = [], []
    kinds = [(("aos", 0), ("soa", 0)), (("soa", 0), ("aosoa", 128)), (("aosoa", 32), ("aos", 0)),
             (("soa", 0), ("aos", 0))]
    for j, n in enumerate([1, 31, 32, 33, 511, 513, 544, 545, 1151, 1152, 1153, 4097, 20000]):
        for name in ("cells", "points"):
            desc = datagen.WORKLOAD_SCHEMAS[name]
            s, o = mrn.Schema(desc), oracle.Schema(desc)
            (sk, sb), (dk, db) = kinds[(j + len(name)) % len(kinds)]
            d = datagen.workload(name, n, 700 + j)
            o_src = oracle.pack(o, d, sk, sb)
            want = oracle.convert(o, o_src, dk, db).base
            dst = dev_dest(s, dk, n, 0, db)
            pairs.append((mrn.View(s, sk, n, block=sb, base=dev(o_src.base)), dst))
            checks.append((dst, want))
    b = mrn.Batch(pairs, use_graph=True)
    b.launch()
    assert mrn.sync() == mrn.OK
    for k, (dst, want) in enumerate(checks):
        assert np.array_equal(host(dst.tensors[0], want.size), want), "job %d" % k


def test_batch_tune_keeps_results_exact():
    """The batch autotuner times launch shapes on the batch's own jobs; the
    tuned batch (re-captured graph) still gives the oracle's bytes."""
    jobs = make_jobs(11, 24)
    b = mrn.Batch([(s, d) for s, d, _, _ in jobs], use_graph=True)
    r = b.tune()
    # the tuned shape is one of the candidates, or the default when that was fastest
    assert 1 <= r["max_chunk"] <= 16 and r["ctas_per_sm"] in (0, 2)
    assert 0 < r["ms"] <= r["default_ms"] <= r["worst_ms"] and r["candidates"] == 11
    for _, d, _, _ in jobs:
        d.tensors[0].fill_(0xA5)
        if d.tensors[1] is not None:
            d.tensors[1].fill_(0xA5)
    b.launch()
    assert mrn.sync() == mrn.OK
    for i, (s, d, want, name) in enumerate(jobs):
        assert np.array_equal(result(d, want, name), want), "job %d (%s)" % (i, name)


def test_jagged_aosoa_jobs_in_a_batch():
    """Jagged AoS -> AoSoA(B) and AoSoA(B) -> AoS jobs in one launch equal
    the oracle; a field-major to field-major jagged job is refused."""
    pairs, checks = [], []
    for j, (n, B) in enumerate([(777, 32), (5000, 128), (513, 5), (20000, 32)]):
        s, o = mrn.Schema(datagen.TRACKS), oracle.Schema(datagen.TRACKS)
        d = datagen.workload("tracks", n, 800 + j)
        o_aos = oracle.pack(o, d, "aos")
        o_blk = oracle.convert(o, o_aos, "aosoa", B, m=d["m"])
        dst = dev_dest(s, "aosoa", n, d["m"], B)
        pairs.append((mrn.View(s, "aos", n, base=dev(o_aos.base), child_pool=dev(o_aos.pool), m=d["m"]), dst))
        checks.append((dst.tensors[0], o_blk.base[: o.base_bytes("aosoa", B, n, d["m"])]))
        back = dev_dest(s, "aos", n, d["m"])
        pairs.append((mrn.View(s, "aosoa", n, block=B, base=dev(o_blk.base), m=d["m"]), back))
        checks.append((back.tensors[0], o_aos.base[: n * 24]))
        checks.append((back.tensors[1], o_aos.pool[: d["m"] * 8]))
    b = mrn.Batch(pairs, use_graph=True)
    b.launch()
    assert mrn.sync() == mrn.OK
    for k, (t, want) in enumerate(checks):
        assert np.array_equal(host(t, want.size), want), "check %d" % k
    s = mrn.Schema(datagen.TRACKS)
    a = mrn.View(s, "soa", 10, base=garbage(1 << 12), m=1)
    c = mrn.View(s, "aosoa", 10, block=32, base=garbage(1 << 12), m=1)
    with pytest.raises(mrn.MrnError):
        mrn.Batch([(a, c)], use_graph=False)


def test_empty_jobs_in_a_batch():
    """Collections of zero objects in a batch: a jagged AoS -> SoA job still
    writes its single offset (0), the others write nothing, and the jobs
    around them are unaffected."""
    jobs = make_jobs(31, 6)
    for name in ("tracks", "cells", "points"):
        desc = datagen.WORKLOAD_SCHEMAS[name]
        s, o = mrn.Schema(desc), oracle.Schema(desc)
        d = datagen.workload(name, 0, 5)
        o_src = oracle.pack(o, d, "aos")
        dk = "soa" if name != "points" else "aosoa"
        o_dst = oracle.convert(o, o_src, dk, 32 if dk == "aosoa" else 0, m=0)
        src = mrn.View(s, "aos", 0, base=dev(o_src.base), child_pool=dev(o_src.pool) if name == "tracks" else None)
        dst = dev_dest(s, dk, 0, 0, 32 if dk == "aosoa" else 0)
        # only the layout's own bytes (none for a plain empty collection)
        jobs.append((src, dst, o_dst.base[: s.required_bytes(dk, 0, 0, 32 if dk == "aosoa" else 0)], name))
    jobs += make_jobs(32, 6)
    for use_graph in (True, False):
        for _, d, _, _ in jobs:
            d.tensors[0].fill_(0xA5)
        b = mrn.Batch([(s, d) for s, d, _, _ in jobs], use_graph=use_graph)
        b.launch()
        assert mrn.sync() == mrn.OK
        for i, (s, d, want, name) in enumerate(jobs):
            assert np.array_equal(result(d, want, name), want), "job %d (%s)" % (i, name)


@pytest.mark.usefixtures("jagged_path")
def test_mixed_size_law_batch_matches_oracle_with_timed_launch():
    """320 collections drawn as in the 4,096-collection mixed batch (seed 3:
    records round(10^U(3, 6)), schema uniform over points / cells / tracks,
    AoS source, target uniform over SoA / AoSoA(32) / AoSoA(128)), each
    size capped at 10,000 records so the oracle runs in seconds.  The plain
    replay and the timed replay (events recorded after the jagged tiles)
    both give the oracle's bytes, and the events measure both parts."""
    t = torch_mod()
    rng = np.random.default_rng(3)
    count = 320
    ns = np.rint(10.0 ** rng.uniform(3.0, 6.0, count)).astype(np.int64)
    sch = rng.integers(0, 3, count)
    tgt = rng.integers(0, 3, count)
    targets = [("soa", 0), ("aosoa", 32), ("aosoa", 128)]
    pairs, checks = [], []
    schemas = {k: (mrn.Schema(datagen.WORKLOAD_SCHEMAS[k]), oracle.Schema(datagen.WORKLOAD_SCHEMAS[k]))
               for k in NAMES}
    for j in range(count):
        name, n = NAMES[sch[j]], int(min(ns[j], 10000))
        dk, db = targets[tgt[j]]
        s, o = schemas[name]
        d = datagen.workload(name, n, 3000 + j)
        o_aos = oracle.pack(o, d, "aos")
        m = d["m"] if name == "tracks" else 0
        want = oracle.convert(o, o_aos, dk, db, m=m).base[: o.base_bytes(dk, db, n, m)]
        pool = dev(o_aos.pool) if name == "tracks" else None
        src = mrn.View(s, "aos", n, base=dev(o_aos.base), child_pool=pool, m=m)
        dst = dev_dest(s, dk, n, m, db)
        pairs.append((src, dst))
        checks.append((dst, want))
    b = mrn.Batch(pairs, use_graph=True)
    ev = [t.cuda.Event(enable_timing=True) for _ in range(3)]
    for timed in (False, True, True):
        for dst, _ in checks:
            dst.tensors[0].fill_(0xA5)
        if timed:
            b.launch_timed(*ev)
        else:
            b.launch()
        assert mrn.sync() == mrn.OK
        for k, (dst, want) in enumerate(checks):
            assert np.array_equal(host(dst.tensors[0], want.size), want), "job %d (timed %s)" % (k, timed)
    t.cuda.synchronize()
    assert ev[0].elapsed_time(ev[1]) > 0 and ev[1].elapsed_time(ev[2]) > 0


def torch_mod():
    import torch
    return torch


def test_timed_launch_with_fresh_events_each_time():
    """mrn_batch_launch_timed points the graph's three event-record nodes at
    the caller's events on every call.  Events destroyed after one call and
    created anew for the next may reuse the addresses the nodes still name;
    the call must still succeed, measure, and give the oracle's bytes.
    Repeated events are refused."""
    import gc
    t = torch_mod()
    jobs = make_jobs(41, 12)
    b = mrn.Batch([(s, d) for s, d, _, _ in jobs], use_graph=True)
    for rnd in range(8):
        ev = [t.cuda.Event(enable_timing=True) for _ in range(3)]
        for _, d, _, _ in jobs:
            d.tensors[0].fill_(0xA5)
        b.launch_timed(*ev)
        assert mrn.sync() == mrn.OK
        t.cuda.synchronize()
        assert ev[0].elapsed_time(ev[2]) > 0, "round %d" % rnd
        for i, (s, d, want, name) in enumerate(jobs):
            assert np.array_equal(result(d, want, name), want), "round %d job %d" % (rnd, i)
        del ev
        gc.collect()
    e = t.cuda.Event(enable_timing=True)
    e.record()
    with pytest.raises(mrn.MrnError):
        b.launch_timed(e, e, t.cuda.Event(enable_timing=True))


def test_narrow_records_in_a_batch():
    """Records of one 4-byte column and of two 2-byte columns, which single
    conversions move by their own tile paths, take the general staged body in
    the persistent batch kernel: both directions, tile edges, one launch,
    each equal to the oracle."""
    pairs, checks = [], []
    for desc in ([("x", "f32", 1)], [("t", "u16", 1), ("adc", "u16", 1)]):
        s, o = mrn.Schema(desc), oracle.Schema(desc)
        for j, n in enumerate([1, 33, 3072 * 2 + 96, 100003]):
            d = datagen.random_columns(desc, n, 90 + j)
            for sk, dk in (("aos", "soa"), ("soa", "aos")):
                o_src = oracle.pack(o, d, sk)
                want = oracle.convert(o, o_src, dk).base
                dst = dev_dest(s, dk, n)
                pairs.append((mrn.View(s, sk, n, base=dev(o_src.base)), dst))
                checks.append((dst, want))
    b = mrn.Batch(pairs, use_graph=True)
    b.launch()
    assert mrn.sync() == mrn.OK
    for k, (dst, want) in enumerate(checks):
        assert np.array_equal(host(dst.tensors[0], want.size), want), "job %d" % k


@pytest.mark.parametrize("case", ["canonical", "swapped_runs", "extra_records", "shuffled", "late_break"])
def test_batch_pool_checks(case, jagged_path):
    """A batched jagged job's pool is converted as one plain conversion
    only when canonical: swapped runs, records beyond the children, a
    shuffled pool and a break in the last parents tile take the fall-back
    pass.  Offsets and child rows equal the oracle's, child rows past the
    written count (capacity above the pool) keep their bytes, and a plain
    job beside it is exact."""
    n = 9 * 1024 + 333
    s, o = mrn.Schema(datagen.TRACKS), oracle.Schema(datagen.TRACKS)
    d = datagen.workload("tracks", n, 71)
    o_aos = oracle.pack(o, d, "aos")
    m, lens = d["m"], d["lengths"]
    if case in ("swapped_runs", "late_break"):
        order = np.arange(n)
        lo, hi = (2048, 3072) if case == "swapped_runs" else (n - 40, n)
        nz = [i for i in range(lo, hi) if lens[i] > 0]
        order[nz[1]], order[nz[2]] = nz[2], nz[1]
        o_aos = oracle.shuffle_pool(o, o_aos, order, gap=0)
    elif case == "extra_records":
        pool = np.concatenate([o_aos.pool[: m * 8], np.full(50 * 8, 7, np.uint8)])
        o_aos = oracle.Side("aos", n, m + 50, base=o_aos.base, pool=pool)
    elif case == "shuffled":
        o_aos = oracle.shuffle_pool(o, o_aos, np.random.default_rng(5).permutation(n), gap=0)
    cap = o_aos.m + 100
    o_soa = oracle.convert(o, o_aos, "soa", m=m)
    cols = [garbage(n * 4) for _ in range(3)]
    offs = garbage((n + 1) * 4)
    kids = [garbage(cap * 4) for _ in range(2)]
    dst = mrn.View(s, "soa", n, columns=cols, offsets=offs, child_columns=kids, m=cap)
    src = mrn.View(s, "aos", n, base=dev(o_aos.base), child_pool=dev(o_aos.pool), m=o_aos.m)
    c_s, c_o = mrn.Schema(datagen.CELLS), oracle.Schema(datagen.CELLS)
    cd = datagen.workload("cells", 7000, 72)
    c_src = oracle.pack(c_o, cd, "aos")
    c_dst = dev_dest(c_s, "soa", 7000)
    b = mrn.Batch([(src, dst), (mrn.View(c_s, "aos", 7000, base=dev(c_src.base)), c_dst)], use_graph=True)
    for _ in range(2):
        for t in cols + [offs] + kids:
            t.fill_(0xA5)
        b.launch()
        assert mrn.sync() == mrn.OK
        for c in range(3):
            assert np.array_equal(host(cols[c]), oracle.region(o, o_soa, c))
        assert np.array_equal(host(offs), oracle.region(o, o_soa, 3))
        for c in range(2):
            got = host(kids[c])
            assert np.array_equal(got[: m * 4], oracle.region(o, o_soa, 4 + c)), "child column %d" % c
            assert (got[m * 4:] == 0xA5).all(), "child rows past the count were written"
        want = oracle.convert(c_o, c_src, "soa").base
        assert np.array_equal(host(c_dst.tensors[0], want.size), want)


def test_batch_offset_base_forms(jagged_path):
    """offset_base in a batch: a canonical pool with a base (the local form
    writes base + the begins), a shard whose begins start inside a larger
    pool (the local check fails: the fused fall-back writes the offsets),
    and a base whose u32 offsets overflow (no local form: the fused job
    records MRN_EOVERFLOW); the first two equal the oracle's offsets plus
    their base, with the oracle's children."""
    s, o = mrn.Schema(datagen.TRACKS), oracle.Schema(datagen.TRACKS)
    d = datagen.workload("tracks", 6000, 81)
    o_aos = oracle.pack(o, d, "aos")
    o_soa = oracle.convert(o, o_aos, "soa", m=d["m"])
    whole_off = oracle.region(o, o_soa, 3).view(np.uint32).astype(np.uint64)
    lens = d["lengths"]
    half = 2500
    m0, m1 = int(lens[:half].sum()), int(lens[half:].sum())
    pairs, checks = [], []
    # 1. the first shard, its own canonical pool, base 123,456
    sub = oracle.Side("aos", half, m0, base=o_aos.base[: half * 24].copy(), pool=o_aos.pool[: m0 * 8].copy())
    want1 = oracle.convert(o, sub, "soa", m=m0)
    offs1, kids1 = garbage((half + 1) * 4), [garbage(m0 * 4) for _ in range(2)]
    cols1 = [garbage(half * 4) for _ in range(3)]
    pairs.append((mrn.View(s, "aos", half, base=dev(sub.base), child_pool=dev(sub.pool), m=m0),
                  mrn.View(s, "soa", half, columns=cols1, offsets=offs1, child_columns=kids1, m=m0,
                           offset_base=123456)))
    # 2. the second shard, begins from m0 in the whole pool, base m0 (a child
    #    capacity of the whole pool, so that a batch may run it split)
    n2 = 6000 - half
    pairs.append((mrn.View(s, "aos", n2, base=dev(o_aos.base[half * 24: 6000 * 24].copy()),
                           child_pool=dev(o_aos.pool), m=o_aos.m),
                  None))
    offs2, kids2 = garbage((n2 + 1) * 4), [garbage(o_aos.m * 4) for _ in range(2)]
    cols2 = [garbage(n2 * 4) for _ in range(3)]
    pairs[-1] = (pairs[-1][0], mrn.View(s, "soa", n2, columns=cols2, offsets=offs2, child_columns=kids2,
                                        m=o_aos.m, offset_base=m0))
    # 3. a base that overflows u32 offsets
    d3 = datagen.workload("tracks", 600, 82)
    o3 = oracle.pack(o, d3, "aos")
    dst3 = dev_dest(s, "soa", 600, d3["m"])
    dst3.s.offset_base = 2**32 - 100
    pairs.append((mrn.View(s, "aos", 600, base=dev(o3.base), child_pool=dev(o3.pool), m=d3["m"]), dst3))
    b = mrn.Batch(pairs, use_graph=True)
    for _ in range(2):
        b.launch()
        bits = mrn.sync_bits()
        assert bits & (1 << mrn.EOVERFLOW) and not bits & ~(1 << mrn.EOVERFLOW)
        got1 = host(offs1).view(np.uint32).astype(np.uint64)
        assert np.array_equal(got1, oracle.region(o, want1, 3).view(np.uint32).astype(np.uint64) + 123456)
        for c in range(2):
            assert np.array_equal(host(kids1[c]), oracle.region(o, want1, 4 + c))
        for c in range(3):
            assert np.array_equal(host(cols1[c]), oracle.region(o, want1, c))
            assert np.array_equal(host(cols2[c]), oracle.region(o, o_soa, c)[half * 4:])
        got2 = host(offs2).view(np.uint32).astype(np.uint64)
        assert np.array_equal(got2, whole_off[half:])
        for c in range(2):
            assert np.array_equal(host(kids2[c], m1 * 4), oracle.region(o, o_soa, 4 + c)[m0 * 4:])
