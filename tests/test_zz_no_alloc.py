"""The allocation-free jagged conversion (mrn_convert_jagged_noalloc).

Callers that cannot let a library allocate device memory (their own pool
owns the GPU, the device is nearly full, or an allocator call is too slow
for their loop) use this entry point; its scan scratch is a fixed array in
the library.  Its output must equal the oracle's and mrn_convert's, byte for
byte, on two calls in a row (the second call reuses the array the first one
left behind).  This file is collected last so that a run stopping at the
first failure has run every other test already.
"""
import os
import re

import numpy as np
import pytest

import datagen
import oracle
import paper_2511_04853_b300 as mrn
from gpu_util import garbage, dev, host, torch

pytestmark = pytest.mark.gpu

_CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2511_04853_b300", "csrc")


def _define(fname, name):
    with open(os.path.join(_CSRC, fname)) as f:
        m = re.search(r"#define\s+%s\s+\(?(\d+)u?\s*(?:\*\s*(\d+)u?)?\)?" % name, f.read())
    assert m, "%s not found in %s" % (name, fname)
    return int(m.group(1)) * (int(m.group(2)) if m.group(2) else 1)


def max_parents():
    """Parents one call may convert: the array holds a 256-byte counter
    block and one 8-byte look-back word per tile of MRN_JAG_TILE parents."""
    tile = _define("mrn_plan.h", "MRN_JAG_TILE")
    scratch = _define("mrn_noalloc.cu", "MRN_NOALLOC_SCRATCH_BYTES")
    return (scratch - 256) // 8 * tile


def _call(src, dst):
    return mrn.lib().mrn_convert_jagged_noalloc(src.ref, dst.ref, mrn.mrn._stream(None))


@pytest.mark.parametrize("n,seed", [(100000, 2), (257, 5)])
def test_matches_oracle_and_mrn_convert_twice(n, seed):
    s, o = mrn.Schema(datagen.TRACKS), oracle.Schema(datagen.TRACKS)
    for call in range(2):
        d = datagen.workload("tracks", n, seed + call)
        o_aos = oracle.pack(o, d, "aos")
        want_o = oracle.convert(o, o_aos, "soa")
        src = mrn.View(s, "aos", n, base=dev(o_aos.base), child_pool=dev(o_aos.pool), m=d["m"])
        nb = s.required_bytes("soa", n, d["m"])
        want_t, got_t = garbage(nb), garbage(nb)
        mrn.convert(src, mrn.View(s, "soa", n, base=want_t, m=d["m"]))
        assert mrn.sync() == mrn.OK
        assert _call(src, mrn.View(s, "soa", n, base=got_t, m=d["m"])) == mrn.OK
        assert mrn.sync() == mrn.OK
        got = host(got_t)
        assert np.array_equal(got[: want_o.base.size], want_o.base), "call %d differs from the oracle" % call
        assert np.array_equal(got, host(want_t)), "call %d differs from mrn_convert" % call


def test_limit_is_accepted_and_one_more_is_refused():
    """At exactly the array's limit the call runs and equals mrn_convert;
    one parent more is refused before anything runs.  The views are backed
    by buffers of the size they describe (every length 0), so a check that
    let an over-size call through would fail this test, never access memory
    outside its buffers."""
    t = torch()
    s = mrn.Schema(datagen.TRACKS)
    lim = max_parents()
    for n, want in ((lim, mrn.OK), (lim + 1, mrn.ESIZE)):
        aos = t.zeros(s.required_bytes("aos", n, 1), dtype=t.uint8, device="cuda")
        pool = t.zeros(s.child_pool_bytes(1), dtype=t.uint8, device="cuda")
        got = garbage(s.required_bytes("soa", n, 1))
        src = mrn.View(s, "aos", n, base=aos, child_pool=pool, m=1)
        assert _call(src, mrn.View(s, "soa", n, base=got, m=1)) == want
        assert mrn.sync() == mrn.OK
        if want == mrn.OK:
            ref = garbage(got.numel())
            mrn.convert(src, mrn.View(s, "soa", n, base=ref, m=1))
            assert mrn.sync() == mrn.OK
            assert t.equal(got, ref), "the call at the limit differs from mrn_convert"
            del ref
        del aos, pool, got
    buf = garbage(1 << 12)
    c = mrn.Schema(datagen.CELLS)
    assert _call(mrn.View(c, "aos", 10, base=buf), mrn.View(c, "soa", 10, base=buf)) == mrn.EINVAL
