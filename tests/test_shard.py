"""Sharding of one collection over ranks: record ranges (aligned, disjoint,
covering), the exchange of per-rank child counts (one all-gather over a
gloo process group of CPU ranks), and, on the GPU, per-range conversions
with ``offset_base`` that concatenate to the whole collection's result
(Sec. V, jagged vector property: the offsets are the prefix sum of the
sizes, so a rank's offsets start at the children of all earlier ranks)."""
import os
import socket

import numpy as np
import pytest

import datagen
import oracle
from paper_2511_04853_b300 import shard


@pytest.mark.parametrize("n", [0, 1, 255, 256, 257, 1000, 4096, 100003])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
@pytest.mark.parametrize("align", [1, 32, 256, 384])
def test_ranges_cover_disjoint_aligned_balanced(n, world, align):
    rs = [shard.shard_range(n, r, world, align) for r in range(world)]
    assert rs[0][0] == 0 and rs[-1][1] == n
    for (lo, hi), (lo2, _) in zip(rs, rs[1:]):
        assert lo <= hi == lo2
    for lo, hi in rs:
        assert lo % align == 0 or lo == n
    units = [-(-(hi - lo) // align) for lo, hi in rs]
    assert max(units) - min(units) <= 1


def test_alignment_and_bases():
    assert shard.alignment(32, 128, 0, None, 384) == 384
    assert shard.alignment() == 1
    assert shard.alignment(5, 32) == 160
    assert shard.exclusive_bases([3, 0, 7, 1]) == ([0, 3, 3, 10], 11)
    with pytest.raises(ValueError):
        shard.shard_range(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n, align):
    """One CPU rank: converts its record range with the oracle, exchanges
    its child count, offsets its offsets by the base and checks its part of
    the whole collection's result."""
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        o = oracle.Schema(datagen.TRACKS)
        d = datagen.workload("tracks", n, 21, mean_len=3.0)
        whole_aos = oracle.pack(o, d, "aos")
        whole = oracle.convert(o, whole_aos, "soa", m=d["m"])
        lo, hi = shard.shard_range(n, rank, world, align)
        sub = oracle.Side("aos", hi - lo, whole_aos.m, base=whole_aos.base[lo * 24: hi * 24].copy(),
                          pool=whole_aos.pool)
        m_local = int(d["lengths"][lo:hi].sum())
        part = oracle.convert(o, sub, "soa", m=m_local)
        base, total = shard.child_base(m_local)
        assert total == d["m"]
        assert base == int(d["lengths"][:lo].sum())
        offs = oracle.region(o, part, 3).view(np.uint32).astype(np.int64) + base
        want_offs = oracle.region(o, whole, 3).view(np.uint32).astype(np.int64)[lo: hi + 1]
        assert np.array_equal(offs, want_offs)
        for c in range(2):
            got = oracle.region(o, part, 4 + c)
            want = oracle.region(o, whole, 4 + c)[base * 4: (base + m_local) * 4]
            assert np.array_equal(got, want)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n,align", [(2, 5003, 256), (3, 300, 256), (2, 0, 1)])
def test_gloo_ranks_concatenate_to_whole(world, n, align):
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(world, _free_port(), n, align), nprocs=world, join=True)


@pytest.mark.gpu
@pytest.mark.parametrize("world", [2, 3])
def test_gpu_ranges_with_offset_base_concatenate(world):
    """The per-rank conversions of a replica run, one after another on one
    GPU (they never wait on each other): child counts from the library's
    count kernel, bases by the exclusive scan, offsets made global by
    offset_base; the concatenation equals the oracle's whole result."""
    import paper_2511_04853_b300 as mrn
    from gpu_util import dev, garbage, host
    n = 7001
    s, o = mrn.Schema(datagen.TRACKS), oracle.Schema(datagen.TRACKS)
    d = datagen.workload("tracks", n, 22)
    o_aos = oracle.pack(o, d, "aos")
    whole = oracle.convert(o, o_aos, "soa", m=d["m"])
    pool = dev(o_aos.pool)
    ranges = [shard.shard_range(n, r, world, shard.alignment(256)) for r in range(world)]
    srcs, counts = [], []
    for lo, hi in ranges:
        v = mrn.View(s, "aos", hi - lo, base=dev(o_aos.base[lo * 24: hi * 24].copy()), child_pool=pool,
                     m=o_aos.m)
        srcs.append(v)
        counts.append(mrn.jagged_count(v))
    bases, total = shard.exclusive_bases(counts)
    assert total == d["m"]
    offs_parts, kid_parts = [], [[], []]
    for (lo, hi), v, base, mm in zip(ranges, srcs, bases, counts):
        offs = garbage((hi - lo + 1) * 4)
        kids = [garbage(max(1, mm) * 4) for _ in range(2)]
        cols = [garbage(max(1, hi - lo) * 4) for _ in range(3)]
        dst = mrn.View(s, "soa", hi - lo, columns=cols, offsets=offs, child_columns=kids, m=mm, offset_base=base)
        mrn.convert(v, dst)
        assert mrn.sync() == mrn.OK
        offs_parts.append(host(offs).view(np.uint32))
        for c in range(2):
            kid_parts[c].append(host(kids[c])[: mm * 4])
    offs_all = np.concatenate([p[:-1] for p in offs_parts[:-1]] + [offs_parts[-1]])
    assert np.array_equal(offs_all, oracle.region(o, whole, 3).view(np.uint32))
    for c in range(2):
        assert np.array_equal(np.concatenate(kid_parts[c]), oracle.region(o, whole, 4 + c))
