"""GPU tests of the continuous-batching server: every request's result equals
the oracle and is the same alone and in a mix of concurrent requests;
admission respects the HBM budget (over-budget requests are rejected, the
rest queue until memory frees); tickets behave."""
import numpy as np
import pytest

import datagen
import oracle
import paper_2511_04853_b300 as mrn
from gpu_util import dev, garbage, host, torch

pytestmark = pytest.mark.gpu


def pinned_from(arr):
    a = np.ascontiguousarray(arr).view(np.uint8).reshape(-1)
    if a.size == 0:
        a = np.zeros(1, np.uint8)
    return torch().from_numpy(a.copy()).pin_memory()


def pinned(nbytes):
    return torch().full((max(1, int(nbytes)),), 0xA5, dtype=torch().uint8).pin_memory()


class Req:
    """One request: source/destination views over host or device buffers,
    and the oracle's expected destination bytes."""

    def __init__(self, rng, idx):
        name = ["points", "cells", "tracks"][idx % 3]
        desc = datagen.WORKLOAD_SCHEMAS[name]
        self.s, self.o = mrn.Schema(desc), oracle.Schema(desc)
        n = int(10 ** rng.uniform(2, 4.7))
        d = datagen.workload(name, n, 100 + idx)
        mode = ["h2d", "d2h", "h2h"][rng.integers(0, 3)]
        self.mode, self.name, self.n = mode, name, n
        if name == "tracks":
            m = d["m"]
            o_aos = oracle.pack(self.o, d, "aos")
            o_soa = oracle.convert(self.o, o_aos, "soa", m=m)
            if mode == "d2h":
                self.src_bufs = (dev(o_soa.base),)
                self.src = mrn.View(self.s, "soa", n, base=self.src_bufs[0], m=m)
                self.dst_bufs = (pinned(n * 24), pinned(m * 8))
                self.dst = mrn.View(self.s, "aos", n, base=self.dst_bufs[0], child_pool=self.dst_bufs[1], m=m,
                                    mem="pinned")
                self.want = np.concatenate([o_aos.base[: n * 24], o_aos.pool[: m * 8]])
            else:
                self.src_bufs = (pinned_from(o_aos.base), pinned_from(o_aos.pool))
                self.src = mrn.View(self.s, "aos", n, base=self.src_bufs[0], child_pool=self.src_bufs[1], m=m,
                                    mem="pinned")
                nb = self.s.required_bytes("soa", n, m)
                self.dst_bufs = (pinned(nb),) if mode == "h2h" else (garbage(nb),)
                self.dst = mrn.View(self.s, "soa", n, base=self.dst_bufs[0], m=m,
                                    mem="pinned" if mode == "h2h" else "device")
                self.want = o_soa.base
        else:
            kinds = [("aos", 0), ("soa", 0), ("aosoa", 32), ("aosoa", 128)]
            sk, sb = kinds[rng.integers(0, 4)]
            dk, db = kinds[rng.integers(0, 4)]
            o_src = oracle.pack(self.o, d, sk, sb)
            o_dst = oracle.convert(self.o, o_src, dk, db)
            src_dev, dst_dev = mode == "d2h", mode == "h2d"
            self.src_bufs = (dev(o_src.base) if src_dev else pinned_from(o_src.base),)
            nb = self.s.required_bytes(dk, n, 0, db)
            self.dst_bufs = (garbage(nb) if dst_dev else pinned(nb),)
            self.src = mrn.View(self.s, sk, n, block=sb, base=self.src_bufs[0],
                                mem="device" if src_dev else "pinned")
            self.dst = mrn.View(self.s, dk, n, block=db, base=self.dst_bufs[0],
                                mem="device" if dst_dev else "pinned")
            self.want = o_dst.base

    def result(self):
        if self.name == "tracks" and self.mode == "d2h":
            return np.concatenate([self.dst_bufs[0].numpy()[: self.n * 24],
                                   self.dst_bufs[1].numpy()[: self.dst.s.n_children * 8]])
        b = self.dst_bufs[0]
        a = b.cpu().numpy() if b.is_cuda else b.numpy()
        return a[: self.want.size]

    def reset(self):
        for b in self.dst_bufs:
            b.fill_(0xA5)


def test_each_result_same_alone_and_in_the_mix():
    rng = np.random.default_rng(3)
    reqs = [Req(rng, i) for i in range(24)]
    sv = mrn.Server(512 << 20, max_slots=4, chunk_bytes=256 << 10)
    try:
        # the mix: everything submitted at once, overlapping on the device
        tickets = []
        for r in reqs:
            rc, t = sv.submit(r.src, r.dst)
            assert rc == mrn.OK
            tickets.append(t)
        for t in tickets:
            assert sv.wait(t, 120.0) == mrn.OK
        torch().cuda.synchronize()
        mixed = [r.result().copy() for r in reqs]
        for r, got in zip(reqs, mixed):
            assert np.array_equal(got, r.want), (r.name, r.mode)
        # alone: one request at a time
        for r, got in zip(reqs, mixed):
            r.reset()
            rc, t = sv.submit(r.src, r.dst)
            assert rc == mrn.OK and sv.wait(t, 120.0) == mrn.OK
            torch().cuda.synchronize()
            assert np.array_equal(r.result(), got)
        st = sv.stats()
        assert st["completed"] == 48 and st["failed"] == 0 and st["rejected"] == 0
        assert st["p50_ms"] > 0 and st["p99_ms"] >= st["p50_ms"]
        assert st["peak_device_bytes"] <= 512 << 20
    finally:
        sv.close()


def test_budget_admission_and_rejection():
    n = 200000
    s, o = mrn.Schema(datagen.CELLS), oracle.Schema(datagen.CELLS)
    d = datagen.workload("cells", n, 1)
    o_aos = oracle.pack(o, d, "aos")
    want = oracle.convert(o, o_aos, "soa").base
    src = mrn.View(s, "aos", n, base=pinned_from(o_aos.base), mem="pinned")
    budget = 24 << 20
    sv = mrn.Server(budget, max_slots=8, chunk_bytes=1 << 20)
    try:
        # host -> host holds a device copy of the destination (4.8 MB) plus
        # staging: a few fit at once, not all ten
        outs = [pinned(s.required_bytes("soa", n)) for _ in range(10)]
        tickets = []
        for out in outs:
            rc, t = sv.submit(src, mrn.View(s, "soa", n, base=out, mem="pinned"))
            assert rc == mrn.OK
            tickets.append(t)
        for t in tickets:
            assert sv.wait(t, 120.0) == mrn.OK
        for out in outs:
            assert np.array_equal(out.numpy()[: want.size], want)
        st = sv.stats()
        assert 0 < st["peak_device_bytes"] <= budget
        # a request that can never fit the budget is rejected at once
        big = 3_000_000
        bsrc = mrn.View(s, "aos", big, base=pinned(big * 24), mem="pinned")
        bdst = mrn.View(s, "soa", big, base=pinned(s.required_bytes("soa", big)), mem="pinned")
        rc, t = sv.submit(bsrc, bdst)
        assert rc == mrn.ENOMEM and t is None
        assert sv.stats()["rejected"] == 1
    finally:
        sv.close()


def test_tickets_and_poll():
    n = 1000
    s, o = mrn.Schema(datagen.POINTS), oracle.Schema(datagen.POINTS)
    d = datagen.workload("points", n, 5)
    o_aos = oracle.pack(o, d, "aos")
    sv = mrn.Server(64 << 20, max_slots=2)
    try:
        dst = garbage(s.required_bytes("soa", n))
        rc, t = sv.submit(mrn.View(s, "aos", n, base=pinned_from(o_aos.base), mem="pinned"),
                          mrn.View(s, "soa", n, base=dst))
        assert rc == mrn.OK
        done, st = False, None
        for _ in range(2_000_000):
            done, st = sv.poll(t)
            if done:
                break
        assert done and st == mrn.OK
        with pytest.raises(mrn.MrnError):
            sv.poll(t)  # consumed
        torch().cuda.synchronize()
        want = oracle.convert(o, o_aos, "soa").base
        assert np.array_equal(host(dst, want.size), want)
        # device -> device is not a served request
        a = garbage(n * 32)
        rc, _ = sv.submit(mrn.View(s, "aos", n, base=a), mrn.View(s, "soa", n, base=dst))
        assert rc == mrn.EINVAL
    finally:
        sv.close()


def test_destroy_drains_outstanding_requests():
    n = 50000
    s, o = mrn.Schema(datagen.CELLS), oracle.Schema(datagen.CELLS)
    d = datagen.workload("cells", n, 2)
    o_aos = oracle.pack(o, d, "aos")
    src = pinned_from(o_aos.base)
    outs = [garbage(s.required_bytes("aosoa", n, 0, 32)) for _ in range(6)]
    sv = mrn.Server(256 << 20, max_slots=3)
    for out in outs:
        rc, _ = sv.submit(mrn.View(s, "aos", n, base=src, mem="pinned"),
                          mrn.View(s, "aosoa", n, block=32, base=out))
        assert rc == mrn.OK
    sv.close()  # waits for all of them
    torch().cuda.synchronize()
    want = oracle.convert(o, o_aos, "aosoa", 32).base
    for out in outs:
        assert np.array_equal(host(out, want.size), want)


def test_wait_latency_reports_each_request():
    """mrn_server_wait_latency returns the request's status and its latency
    (positive, no larger than the largest latency in the statistics), and
    the result equals the oracle."""
    n = 20000
    s, o = mrn.Schema(datagen.CELLS), oracle.Schema(datagen.CELLS)
    d = datagen.workload("cells", n, 8)
    o_aos = oracle.pack(o, d, "aos")
    want = oracle.convert(o, o_aos, "aosoa", 32).base
    src = pinned_from(o_aos.base)
    sv = mrn.Server(256 << 20, max_slots=4)
    try:
        dsts, tickets = [], []
        for _ in range(6):
            dst = garbage(s.required_bytes("aosoa", n, 0, 32))
            rc, t = sv.submit(mrn.View(s, "aos", n, base=src, mem="pinned"),
                              mrn.View(s, "aosoa", n, block=32, base=dst))
            assert rc == mrn.OK
            dsts.append(dst)
            tickets.append(t)
        lats = []
        for t in tickets:
            st, lat = sv.wait_latency(t, 60.0)
            assert st == mrn.OK and lat is not None and lat > 0
            lats.append(lat)
        stt = sv.stats()
        assert max(lats) <= stt["max_ms"] + 1e-9
        torch().cuda.synchronize()
        for dst in dsts:
            assert np.array_equal(host(dst, want.size), want)
    finally:
        sv.close()
