"""The allocation-free jagged conversion (mrn_convert_jagged_noalloc).

Callers that cannot let a library allocate device memory (their own pool
owns the GPU, the device is nearly full, or an allocator call is too slow
for their loop) use this entry point; its scan scratch is a fixed array in
the library.  Its output must equal mrn_convert's, byte for byte, on two
calls in a row (the second call reuses the array the first one left behind).
This file is collected last so that a run stopping at the first failure has
run every other test already.
"""
import numpy as np
import pytest

import datagen
import oracle
import paper_2511_04853_b300 as mrn
from gpu_util import dev, garbage, host, torch

pytestmark = pytest.mark.gpu


def _call(src, dst):
    return mrn.lib().mrn_convert_jagged_noalloc(src.ref, dst.ref, mrn.mrn._stream(None))


@pytest.mark.parametrize("n,seed", [(100000, 2), (257, 5)])
def test_matches_mrn_convert_twice(n, seed):
    s, o = mrn.Schema(datagen.TRACKS), oracle.Schema(datagen.TRACKS)
    for call in range(2):
        d = datagen.workload("tracks", n, seed + call)
        o_aos = oracle.pack(o, d, "aos")
        src = mrn.View(s, "aos", n, base=dev(o_aos.base), child_pool=dev(o_aos.pool), m=d["m"])
        nb = s.required_bytes("soa", n, d["m"])
        want_t, got_t = garbage(nb), garbage(nb)
        mrn.convert(src, mrn.View(s, "soa", n, base=want_t, m=d["m"]))
        assert mrn.sync() == mrn.OK
        assert _call(src, mrn.View(s, "soa", n, base=got_t, m=d["m"])) == mrn.OK
        assert mrn.sync() == mrn.OK
        assert np.array_equal(host(got_t), host(want_t)), "call %d differs" % call


def test_rejects_sizes_beyond_the_array_and_other_layouts():
    """One parent more than the scratch array holds is refused before
    anything runs.  The views are backed by buffers of the size they
    describe (all lengths 0), so a check that let the call through would
    fail this test, never access memory outside its buffers."""
    t = torch()
    s = mrn.Schema(datagen.TRACKS)
    big = 33_521_664 + 1
    buf = garbage(1 << 12)
    aos = t.zeros(s.required_bytes("aos", big, 1), dtype=t.uint8, device="cuda")
    pool = t.zeros(s.child_pool_bytes(1), dtype=t.uint8, device="cuda")
    soa = t.zeros(s.required_bytes("soa", big, 1), dtype=t.uint8, device="cuda")
    src = mrn.View(s, "aos", big, base=aos, child_pool=pool, m=1)
    dst = mrn.View(s, "soa", big, base=soa, m=1)
    assert _call(src, dst) == mrn.ESIZE  # checked before anything runs
    assert mrn.sync() == mrn.OK
    del aos, pool, soa
    c = mrn.Schema(datagen.CELLS)
    assert _call(mrn.View(c, "aos", 10, base=buf), mrn.View(c, "soa", 10, base=buf)) == mrn.EINVAL
