"""Collections in host memory (MRN_MEM_HOST): their size-changing
operations run on the host, so they are checked here without a GPU against
the oracle's plain definitions (Sec. VI-B: resize, reserve, clear,
shrink_to_fit, erase) laid out by the oracle.  The same operations on device
collections, and insert / assign (conversions), are in the GPU tests."""
import ctypes

import numpy as np
import pytest

import datagen
import oracle
from oracle import collection as oc
import paper_2511_04853_b300 as mrn
from coll_util import contents, expected, fill

LAYOUTS = [("aos", 0), ("soa", 0), ("aosoa", 32), ("aosoa", 7)]


def _pair(name):
    desc = datagen.WORKLOAD_SCHEMAS[name]
    return mrn.Schema(desc), oracle.Schema(desc)


@pytest.mark.parametrize("kind,B", LAYOUTS)
@pytest.mark.parametrize("name", ["cells", "points"])
def test_host_resize_reserve_shrink(name, kind, B):
    s, o = _pair(name)
    d = datagen.workload(name, 300, 3)
    c = mrn.Collection(s, kind, capacity=10, block=B, mem="host")
    fill(c, o, d, kind, B)
    assert contents(c, o) == expected(o, d, kind, B)
    assert c.sizes()[2] >= 300
    c.resize(420)             # grows: all-zero objects at the end
    assert contents(c, o) == expected(o, oc.resize(d, 420), kind, B)
    c.resize(123)             # shrinks (AoSoA: the freed slots are zeroed)
    assert contents(c, o) == expected(o, oc.resize(d, 123), kind, B)
    c.resize(200)             # grows again over zeroed slots
    assert contents(c, o) == expected(o, oc.resize(oc.resize(d, 123), 200), kind, B)
    c.reserve(5000)
    assert c.sizes()[2] == 5000
    assert contents(c, o) == expected(o, oc.resize(oc.resize(d, 123), 200), kind, B)
    c.shrink_to_fit()
    assert c.sizes()[0] == c.sizes()[2] == 200
    assert contents(c, o) == expected(o, oc.resize(oc.resize(d, 123), 200), kind, B)
    c.clear()
    assert c.sizes()[0] == 0


@pytest.mark.parametrize("kind", ["aos", "soa"])
@pytest.mark.parametrize("first,count", [(0, 0), (0, 1), (5, 40), (250, 50), (0, 300), (299, 1), (17, 183)])
def test_host_erase(kind, first, count):
    s, o = _pair("cells")
    d = datagen.workload("cells", 300, 4)
    c = mrn.Collection(s, kind, capacity=300, mem="host")
    fill(c, o, d, kind)
    c.erase(first, count)
    assert c.sizes()[0] == 300 - count
    assert contents(c, o) == expected(o, oc.erase(d, first, count), kind)


def test_host_erase_sequence_and_errors():
    s, o = _pair("points")
    d = datagen.workload("points", 1000, 5)
    c = mrn.Collection(s, "soa", capacity=1000, mem="host")
    fill(c, o, d, "soa")
    rng = np.random.default_rng(0)
    for _ in range(20):
        n = d["n"]
        f = int(rng.integers(0, n + 1))
        k = int(rng.integers(0, min(60, n - f) + 1))
        c.erase(f, k)
        d = oc.erase(d, f, k)
        assert contents(c, o) == expected(o, d, "soa")
    with pytest.raises(mrn.MrnError) as e:
        c.erase(d["n"], 1)
    assert e.value.code == mrn.EINVAL
    blk = mrn.Collection(s, "aosoa", capacity=64, block=32, mem="host")
    blk.resize(40)
    with pytest.raises(mrn.MrnError) as e:
        blk.erase(0, 1)
    assert e.value.code == mrn.EUNSUPPORTED


@pytest.mark.parametrize("src,dst,nbytes", [(100, 0, 1000), (0, 100, 1000), (0, 3, 4093), (7, 0, 64),
                                            (0, 0, 10), (0, 2000, 500)])
def test_host_memmove_overlapping(src, dst, nbytes):
    buf = np.random.default_rng(1).integers(0, 256, 4096 + 2048, dtype=np.uint8)
    want = buf.copy()
    want[dst:dst + nbytes] = buf[src:src + nbytes].copy()
    a = buf.ctypes.data
    mrn.memmove(a + dst, a + src, nbytes, mem="host")
    assert buf.tobytes() == want.tobytes()
