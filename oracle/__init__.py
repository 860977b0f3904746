"""CPU oracle for layout conversion — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import this package.  The conversion library never
does, and this package imports nothing from it.

The arithmetic lives in ``mrn_oracle.c`` (a field-by-field copy per object,
the paper's default transfer, Sec. VI-B "Defining Layouts"); this module
only marshals numpy buffers to it through ctypes.  Helpers that pack
generator values into a layout (:func:`pack`) go through the same C routine,
from per-column arrays.
"""
import ctypes
import os

import numpy as np

from . import build as _build

AOS, SOA, AOSOA = 0, 1, 2
KIND = {"aos": AOS, "soa": SOA, "aosoa": AOSOA}
OK, EINVAL, ESIZE, EOVERFLOW = 0, 1, 2, 4

_SIZES = {"u8": 1, "i8": 1, "bool": 1, "u16": 2, "i16": 2, "u32": 4,
          "i32": 4, "f32": 4, "u64": 8, "i64": 8, "f64": 8}

_lib = None


class _Side(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("block", ctypes.c_uint32),
                ("base", ctypes.c_void_p), ("cols", ctypes.c_void_p),
                ("offsets", ctypes.c_void_p), ("child_cols", ctypes.c_void_p),
                ("pool", ctypes.c_void_p), ("n", ctypes.c_uint64),
                ("m", ctypes.c_uint64), ("gpool", ctypes.c_void_p),
                ("m2", ctypes.c_uint64), ("child_offsets", ctypes.c_void_p),
                ("gchild_cols", ctypes.c_void_p)]


def lib():
    global _lib
    if _lib is None:
        # MRN_ORACLE_LIB lets the mutation test load a deliberately broken
        # copy of this oracle; it is never set otherwise.
        path = os.environ.get("MRN_ORACLE_LIB") or _build.build()
        L = ctypes.CDLL(path)
        vp, u64, u32, i32 = (ctypes.c_void_p, ctypes.c_uint64,
                             ctypes.c_uint32, ctypes.c_int)
        L.orc_schema_new.restype = vp
        L.orc_schema_new.argtypes = [ctypes.POINTER(ctypes.c_int32), i32,
                                     ctypes.POINTER(i32)]
        L.orc_schema_free.argtypes = [vp]
        for name, rt, at in [
                ("orc_ncols", i32, [vp]), ("orc_col_size", u32, [vp, i32]),
                ("orc_col_aos_off", u64, [vp, i32]), ("orc_stride", u64, [vp]),
                ("orc_has_jagged", i32, [vp]), ("orc_len_off", u64, [vp]),
                ("orc_begin_off", u64, [vp]), ("orc_off_size", u32, [vp]),
                ("orc_child", vp, [vp]),
                ("orc_aosoa_col_start", u64, [vp, u32, i32]),
                ("orc_aosoa_block_bytes", u64, [vp, u32]),
                ("orc_soa_region_start", u64, [vp, u64, u64, u64, i32]),
                ("orc_fm_region_start", u64, [vp, i32, u32, u64, u64, u64, i32]),
                ("orc_soa_bytes", u64, [vp, u64, u64, u64]),
                ("orc_base_bytes", u64, [vp, i32, u32, u64, u64, u64]),
                ("orc_col_es", i32, [vp, i32]), ("orc_col_sub", i32, [vp, i32]),
                ("orc_col_store", i32, [vp, i32]), ("orc_nstore", i32, [vp])]:
            f = getattr(L, name)
            f.restype, f.argtypes = rt, at
        L.orc_convert.restype = i32
        L.orc_convert.argtypes = [vp, ctypes.POINTER(_Side),
                                  ctypes.POINTER(_Side),
                                  ctypes.POINTER(ctypes.c_uint64)]
        _lib = L
    return _lib


def tokens(desc):
    """Serialises a schema description (see ``datagen.schemas``) to the
    oracle's token list."""
    out = []
    for m in desc:
        if m[1] == "group":
            out += [2] + tokens(m[2]) + [3]
        elif m[1] == "jagged":
            ch = tokens(m[3])
            out += [4, _SIZES[m[2]], len(ch)] + ch
        elif len(m) > 3 and m[3] == "interleaved":
            out += [5, _SIZES[m[1]], int(m[2])]
        else:
            out += [1, _SIZES[m[1]], int(m[2])]
    return out


class Schema:
    """The oracle's own lowering of a schema description."""

    def __init__(self, desc, _handle=None, _owner=None):
        L = lib()
        self.desc = desc
        self._owner = _owner
        if _handle is None:
            tk = tokens(desc)
            arr = (ctypes.c_int32 * max(1, len(tk)))(*tk)
            st = ctypes.c_int(0)
            h = L.orc_schema_new(arr, len(tk), ctypes.byref(st))
            if not h:
                raise ValueError("oracle rejected schema (status %d)" % st.value)
            self._h = h
        else:
            self._h = _handle
        self.ncols = L.orc_ncols(self._h)
        self.col_size = [L.orc_col_size(self._h, c) for c in range(self.ncols)]
        self.col_aos_off = [L.orc_col_aos_off(self._h, c) for c in range(self.ncols)]
        self.col_es = [L.orc_col_es(self._h, c) for c in range(self.ncols)]
        self.col_sub = [L.orc_col_sub(self._h, c) for c in range(self.ncols)]
        self.col_store = [L.orc_col_store(self._h, c) for c in range(self.ncols)]
        self.nstore = L.orc_nstore(self._h)
        self.stride = L.orc_stride(self._h)
        self.has_jagged = bool(L.orc_has_jagged(self._h))
        self.child = None
        if self.has_jagged:
            self.len_off = L.orc_len_off(self._h)
            self.begin_off = L.orc_begin_off(self._h)
            self.off_size = L.orc_off_size(self._h)
            jm = [m for m in _flat_members(desc) if m[1] == "jagged"][0]
            self.child = Schema(jm[3], _handle=L.orc_child(self._h), _owner=self)

    def __del__(self):
        if self._owner is None and getattr(self, "_h", None) and _lib is not None:
            _lib.orc_schema_free(self._h)
            self._h = None

    # layout rules, as the oracle defines them
    def aosoa_col_start(self, B, c):
        return lib().orc_aosoa_col_start(self._h, B, c)

    def aosoa_block_bytes(self, B):
        return lib().orc_aosoa_block_bytes(self._h, B)

    def soa_region_start(self, n, m, r, m2=0):
        return lib().orc_soa_region_start(self._h, n, m, m2, r)

    def fm_region_start(self, kind, block, n, m, r, m2=0):
        """Start of item r of a single-block field-major side (SoA: data
        columns, offsets, then the child level's items; jagged AoSoA(B):
        blocks, offsets, then the child level's items)."""
        return lib().orc_fm_region_start(self._h, KIND.get(kind, kind), block, n, m, m2, r)

    def base_bytes(self, kind, block, n, m=0, m2=0):
        return lib().orc_base_bytes(self._h, KIND.get(kind, kind), block, n, m, m2)


def _flat_members(desc):
    out = []
    for m in desc:
        out.append(m)
        if m[1] == "group":
            out += _flat_members(m[2])
    return out


def _ptr(a):
    return None if a is None else a.ctypes.data


def _ptr_array(arrs):
    if arrs is None:
        return None, None
    keep = (ctypes.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
    return ctypes.cast(keep, ctypes.c_void_p), keep


class Side:
    """One side of a conversion: numpy buffers in a layout."""

    def __init__(self, kind, n, m=0, block=0, base=None, cols=None,
                 offsets=None, child_cols=None, pool=None, gpool=None, m2=0,
                 child_offsets=None, gchild_cols=None):
        self.kind = KIND.get(kind, kind)
        self.block, self.n, self.m, self.m2 = block, n, m, m2
        self.base, self.cols, self.offsets = base, cols, offsets
        self.child_cols, self.pool, self.gpool = child_cols, pool, gpool
        self.child_offsets, self.gchild_cols = child_offsets, gchild_cols

    def _c(self):
        keep = []
        cols, k1 = _ptr_array(self.cols)
        ccols, k2 = _ptr_array(self.child_cols)
        gcols, k3 = _ptr_array(self.gchild_cols)
        keep += [k1, k2, k3]
        s = _Side(self.kind, self.block, _ptr(self.base), cols,
                  _ptr(self.offsets), ccols, _ptr(self.pool), self.n, self.m,
                  _ptr(self.gpool), self.m2, _ptr(self.child_offsets), gcols)
        return s, keep


def alloc(schema, kind, n, m=0, block=0, m2=0):
    """A zero-filled destination side in single-buffer form."""
    kind = KIND.get(kind, kind)
    base = np.zeros(max(1, schema.base_bytes(kind, block, n, m, m2)), np.uint8)
    pool = gpool = None
    if kind == AOS and schema.has_jagged:
        pool = np.zeros(max(1, m * schema.child.stride), np.uint8)
        if schema.child.has_jagged:
            gpool = np.zeros(max(1, m2 * schema.child.child.stride), np.uint8)
    return Side(kind, n, m, block, base=base, pool=pool, gpool=gpool, m2=m2)


def convert_into(schema, src, dst):
    """Runs the oracle; returns ``(status, m_written)``."""
    cs, k1 = src._c()
    cd, k2 = dst._c()
    mo = ctypes.c_uint64(0)
    st = lib().orc_convert(schema._h, ctypes.byref(cs), ctypes.byref(cd),
                           ctypes.byref(mo))
    del k1, k2
    return st, mo.value


def convert(schema, src, kind, block=0, m=None, m2=None):
    """Converts ``src`` into a freshly allocated side of ``kind``.  For a
    jagged schema ``m`` is the destination's child capacity (default: the
    source's child count), ``m2`` its grandchild capacity for a nested
    member; the number of children written is left in ``.written``."""
    if m is None:
        m = src.m
    if m2 is None:
        m2 = src.m2
    dst = alloc(schema, kind, src.n, m, block, m2)
    st, mo = convert_into(schema, src, dst)
    if st != OK:
        raise ValueError("oracle conversion failed with status %d" % st)
    dst.written = mo
    return dst


def flat_columns(values, interleaved=None):
    """Per-flattened-column arrays from generator leaves (an ``(n, E)`` array
    property becomes E columns).  A leaf marked interleaved stays one
    row-major ``(n, E)`` array; its E column entries are byte views of it
    starting at element k (so that column k's pointer is the array's plus
    k * size), returned with the array that owns them."""
    cols = []
    for i, v in enumerate(values):
        v = np.asarray(v)
        if v.ndim == 1:
            cols.append(np.ascontiguousarray(v).view(np.uint8))
        elif interleaved and interleaved[i]:
            whole = np.ascontiguousarray(v).view(np.uint8).reshape(-1)
            z = v.dtype.itemsize
            for k in range(v.shape[1]):
                cols.append(whole[k * z:])
        else:
            for k in range(v.shape[1]):
                cols.append(np.ascontiguousarray(v[:, k]).view(np.uint8))
    return cols


def _interleaved_flags(desc):
    out = []
    for m in desc:
        if m[1] == "group":
            out += _interleaved_flags(m[2])
        elif m[1] == "jagged":
            continue
        else:
            out.append(len(m) > 3 and m[3] == "interleaved")
    return out


def values_side(schema, data):
    """The generator's values as a per-column SoA side."""
    n = data["n"]
    cols = flat_columns(data["columns"], _interleaved_flags(schema.desc))
    if not cols:
        cols = None
    if not schema.has_jagged:
        return Side(SOA, n, 0, cols=cols, base=np.zeros(1, np.uint8))
    lengths = np.asarray(data["lengths"], dtype=np.uint64)
    offs = np.concatenate([[0], np.cumsum(lengths)]).astype(
        np.uint32 if schema.off_size == 4 else np.uint64)
    jm = [m for m in _flat_members(schema.desc) if m[1] == "jagged"][0]
    kids = flat_columns(data["children"], _interleaved_flags(jm[3]))
    if not schema.child.has_jagged:
        return Side(SOA, n, data["m"], cols=cols, offsets=offs.view(np.uint8),
                    child_cols=kids, base=np.zeros(1, np.uint8))
    # nested: the children's own lengths and the grandchild values
    l1 = np.asarray(data["child_lengths"], dtype=np.uint64)
    offs1 = np.concatenate([[0], np.cumsum(l1)]).astype(
        np.uint32 if schema.child.off_size == 4 else np.uint64)
    gm = [m for m in _flat_members(jm[3]) if m[1] == "jagged"][0]
    grand = flat_columns(data["grandchildren"], _interleaved_flags(gm[3]))
    return Side(SOA, n, data["m"], cols=cols, offsets=offs.view(np.uint8),
                child_cols=kids, base=np.zeros(1, np.uint8), m2=data["m2"],
                child_offsets=offs1.view(np.uint8), gchild_cols=grand)


def pack(schema, data, kind, block=0, pool_perm=None):
    """Generator values laid out in ``kind`` by the oracle.  For a jagged
    schema on the AoS side, ``pool_perm`` (a permutation of the parents)
    reorders the parents' runs in the child pool and rewrites each
    parent's ``begin``."""
    src = values_side(schema, data)
    out = convert(schema, src, kind, block, m=src.m, m2=src.m2)
    if pool_perm is not None and schema.has_jagged and out.kind == AOS:
        out = shuffle_pool(schema, out, pool_perm)
    return out


def shuffle_pool(schema, side, order, gap=0):
    """Re-lays a canonical AoS child pool: parent ``order[k]``'s run of child
    records is placed k-th, with ``gap`` unused (zero) slots before each run;
    every parent's ``begin`` is rewritten to match."""
    n, cs = side.n, schema.child.stride
    rs = schema.stride
    recs = side.base[: n * rs].reshape(n, rs) if n else np.zeros((0, rs), np.uint8)
    lens = [int(recs[i, schema.len_off:schema.len_off + 4].view(np.uint32)[0]) for i in range(n)]
    begs = [int(recs[i, schema.begin_off:schema.begin_off + 8].view(np.uint64)[0]) for i in range(n)]
    m_new = side.m + gap * n
    new_pool = np.zeros(max(1, m_new * cs), np.uint8)
    new_base = side.base.copy()
    cur = 0
    for i in order:
        i = int(i)
        cur += gap
        L, b = lens[i], begs[i]
        new_pool[cur * cs:(cur + L) * cs] = side.pool[b * cs:(b + L) * cs]
        new_base[i * rs + schema.begin_off:i * rs + schema.begin_off + 8] = \
            np.array([cur], np.uint64).view(np.uint8)
        cur += L
    return Side(AOS, n, m_new, base=new_base, pool=new_pool)


def region(schema, side, r):
    """Bytes of region ``r`` of a single-block field-major side: SoA data
    column / offsets / child column, or (jagged AoSoA) blocks / offsets /
    child column."""
    n, m = side.n, side.m
    P = 1 if side.kind == AOSOA else schema.ncols
    start = schema.fm_region_start(side.kind, side.block, n, m, r)
    if r < P:
        size = ((n + side.block - 1) // side.block * schema.aosoa_block_bytes(side.block)
                if side.kind == AOSOA else n * schema.col_size[r])
    elif schema.has_jagged and r == P:
        size = (n + 1) * schema.off_size
    else:
        size = m * schema.child.col_size[r - P - 1]
    return side.base[start:start + size]


def library_path():
    return os.path.abspath(_build.LIB)
