"""Helpers for the collection tests: the regions a collection stores, filled
from and compared with the oracle's layout of the same values."""
import ctypes

import numpy as np

import oracle
import paper_2511_04853_b300 as mrn

KINDS = {"aos": oracle.AOS, "soa": oracle.SOA, "aosoa": oracle.AOSOA}


def _ptrs(arr_ptr, count):
    if not arr_ptr or count == 0:
        return []
    a = ctypes.cast(arr_ptr, ctypes.POINTER(ctypes.c_void_p))
    return [a[i] for i in range(count)]


def regions(coll, o):
    """(address, bytes) of every region holding the collection's n objects
    and m children, in the order ``expected`` lists them."""
    v = coll.view().s
    n, m = v.n_records, v.n_children
    kind, B = v.layout.kind, v.layout.block
    out = []
    if kind == mrn.AOS:
        out.append((v.base, n * o.stride))
        if o.has_jagged:
            out.append((v.child_pool, m * o.child.stride))
        return out
    if kind == mrn.SOA:
        for c, p in enumerate(_ptrs(v.columns, o.ncols)):
            out.append((p, n * o.col_size[c]))
    else:
        out.append((v.base, (n + B - 1) // B * o.aosoa_block_bytes(B) if B else 0))
    if o.has_jagged:
        out.append((v.offsets, (n + 1) * o.off_size))
        for j, p in enumerate(_ptrs(v.child_columns, len(o.child.col_size))):
            out.append((p, m * o.child.col_size[j]))
    return out


def expected(o, data, kind, block=0):
    """The oracle's bytes of those regions for the values ``data``."""
    side = oracle.pack(o, data, kind, block)
    n, m = data["n"], data.get("m", 0)
    if kind == "aos":
        out = [side.base[: n * o.stride]]
        if o.has_jagged:
            out.append(side.pool[: m * o.child.stride])
        return [np.asarray(x).tobytes() for x in out]
    P = 1 if kind == "aosoa" else o.ncols
    count = P + (1 + len(o.child.col_size) if o.has_jagged else 0)
    return [oracle.region(o, side, r).tobytes() for r in range(count)]


def _read(addr, nbytes, mem):
    if nbytes == 0:
        return b""
    if mem == "device":
        import torch
        t = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        mrn.memmove(t, addr, nbytes)
        torch.cuda.synchronize()
        return t.cpu().numpy().tobytes()
    return ctypes.string_at(addr, nbytes)


def _write(addr, data, mem):
    if len(data) == 0:
        return
    if mem == "device":
        import torch
        t = torch.from_numpy(np.frombuffer(data, np.uint8).copy()).cuda()
        mrn.memmove(addr, t, len(data))
        torch.cuda.synchronize()
    else:
        ctypes.memmove(addr, data, len(data))


def fill(coll, o, data, kind, block=0, mem="host"):
    """Sets a collection of a schema without jagged members to the values
    ``data`` by writing the oracle's bytes into its regions (jagged
    collections are filled through ``assign``, which keeps their child count)."""
    assert not o.has_jagged
    coll.resize(data["n"])
    want = expected(o, data, kind, block)
    for (addr, nb), w in zip(regions(coll, o), want):
        assert nb == len(w)
        _write(addr, w, mem)


def contents(coll, o, mem="host"):
    return [_read(a, nb, mem) for a, nb in regions(coll, o)]
