"""Helpers for the GPU parity tests: move oracle-side numpy buffers to the
device, run the library, bring the bytes back."""
import numpy as np

import oracle
import paper_2511_04853_b300 as mrn

GARBAGE = 0xA5  # destinations start filled with this, so unwritten bytes show


def torch():
    import torch as t
    return t


def dev(arr):
    """numpy uint8 buffer -> CUDA uint8 tensor (never empty)."""
    t = torch()
    a = np.ascontiguousarray(arr).view(np.uint8).reshape(-1)
    if a.size == 0:
        a = np.zeros(1, np.uint8)
    return t.from_numpy(a.copy()).cuda()


def garbage(nbytes):
    t = torch()
    return t.full((max(1, int(nbytes)),), GARBAGE, dtype=t.uint8, device="cuda")


def host(tensor, nbytes=None):
    a = tensor.cpu().numpy()
    return a if nbytes is None else a[: int(nbytes)]


def dev_view(schema, side, o_schema):
    """Device copy of an oracle side, as a library view."""
    kind = side.kind
    base = dev(side.base) if side.base is not None else None
    pool = dev(side.pool) if side.pool is not None else None
    v = mrn.View(schema, kind, side.n, block=side.block, base=base, child_pool=pool, m=side.m)
    v.tensors = (base, pool)
    return v


def dev_dest(schema, kind, n, m=0, block=0):
    """A garbage-filled device destination in single-buffer form."""
    base = garbage(schema.required_bytes(kind, n, m, block))
    pool = None
    if kind in ("aos", mrn.AOS) and schema.has_jagged:
        pool = garbage(schema.child_pool_bytes(m))
    v = mrn.View(schema, kind, n, block=block, base=base, child_pool=pool, m=m)
    v.tensors = (base, pool)
    return v


def run(src, dst):
    mrn.convert(src, dst)
    st = mrn.sync()
    assert st == mrn.OK, mrn.status_str(st)


def base_bytes(v, o_schema, kind, n, m=0, block=0):
    return host(v.tensors[0], o_schema.base_bytes(kind, block, n, m))


KINDS = [("aos", 0), ("soa", 0), ("aosoa", 32), ("aosoa", 128), ("aosoa", 8), ("aosoa", 3)]


def oracle_pair(o_schema, data, src_kind, src_block, dst_kind, dst_block, pool_perm=None):
    o_src = oracle.pack(o_schema, data, src_kind, src_block, pool_perm=pool_perm)
    o_dst = oracle.convert(o_schema, o_src, dst_kind, dst_block)
    return o_src, o_dst
