"""ctypes binding of ``libmrn.so`` (declared in ``include/mrn.h``).

Argument marshalling only: every conversion runs in the library's CUDA
kernels.  If the library is missing the import fails loudly; there is no
fallback path.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmrn.so")

OK, EINVAL, ESIZE, EALIGN, EOVERFLOW, ENOMEM, ETIMEOUT, ECUDA, EBUSY, ENOTFOUND, EUNSUPPORTED = range(11)
AOS, SOA, AOSOA = 0, 1, 2
KIND = {"aos": AOS, "soa": SOA, "aosoa": AOSOA}
MEM_HOST, MEM_HOST_PINNED, MEM_DEVICE = 0, 1, 2
MEM = {"host": MEM_HOST, "pinned": MEM_HOST_PINNED, "device": MEM_DEVICE}
DTYPES = {"u8": 0, "i8": 1, "u16": 2, "i16": 3, "u32": 4, "i32": 5, "u64": 6,
          "i64": 7, "f32": 8, "f64": 9, "bool": 10}

vp, u32, u64, i32, sz = (ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64,
                         ctypes.c_int32, ctypes.c_size_t)


class Layout(ctypes.Structure):
    _fields_ = [("kind", i32), ("block", u32)]


class ViewStruct(ctypes.Structure):
    _fields_ = [("schema", vp), ("layout", Layout), ("mem", i32), ("device", i32),
                ("n_records", u64), ("n_children", u64), ("base", vp),
                ("columns", vp), ("offsets", vp), ("child_columns", vp),
                ("child_pool", vp), ("offset_base", u64), ("n_grandchildren", u64),
                ("grandchild_pool", vp)]


class SchemaInfo(ctypes.Structure):
    _fields_ = [("n_columns", u32), ("aos_stride", u32), ("aos_align", u32),
                ("has_jagged", i32), ("jag_length_offset", u32),
                ("jag_begin_offset", u32), ("offset_size", u32),
                ("child_columns", u32), ("child_stride", u32),
                ("reserved", u32), ("hash", u64)]


class ColumnInfo(ctypes.Structure):
    _fields_ = [("size", u32), ("aos_offset", u32), ("dtype", i32),
                ("fm_stride", u32), ("name", ctypes.c_char * 128)]


class TransferOpts(ctypes.Structure):
    _fields_ = [("chunk_bytes", sz), ("n_slots", i32), ("flags", i32)]


class Job(ctypes.Structure):
    _fields_ = [("src", ctypes.POINTER(ViewStruct)), ("dst", ctypes.POINTER(ViewStruct))]


class TuneResult(ctypes.Structure):
    _fields_ = [("threads", u32), ("ctas_per_sm", u32), ("tile_records", u32),
                ("staged", u32), ("gbps", ctypes.c_double),
                ("default_gbps", ctypes.c_double)]


class BatchTuneResult(ctypes.Structure):
    _fields_ = [("max_chunk", u32), ("ctas_per_sm", u32), ("ms", ctypes.c_double),
                ("default_ms", ctypes.c_double), ("worst_ms", ctypes.c_double), ("candidates", u32),
                ("reserved", u32)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", sz), ("max_slots", i32), ("reserved", i32),
                ("chunk_bytes", sz)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", u64), ("admitted", u64), ("completed", u64),
                ("rejected", u64), ("failed", u64), ("bytes_in", u64),
                ("bytes_out", u64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("busy_s", ctypes.c_double),
                ("peak_device_bytes", u64)]


# (name, restype, argtypes) of every exported entry point
SIGNATURES = [
    ("mrn_status_str", ctypes.c_char_p, [ctypes.c_int]),
    ("mrn_version", ctypes.c_int, []),
    ("mrn_schema_create", ctypes.c_int, [ctypes.POINTER(vp)]),
    ("mrn_schema_add_field", ctypes.c_int, [vp, ctypes.c_char_p, ctypes.c_int, u32]),
    ("mrn_schema_add_field_interleaved", ctypes.c_int, [vp, ctypes.c_char_p, ctypes.c_int, u32]),
    ("mrn_required_bytes_nested", ctypes.c_int, [vp, Layout, u64, u64, u64, ctypes.POINTER(sz)]),
    ("mrn_grandchild_pool_bytes", ctypes.c_int, [vp, u64, ctypes.POINTER(sz)]),
    ("mrn_region_offset_nested", ctypes.c_int, [vp, Layout, u64, u64, u64, u32, ctypes.POINTER(sz)]),
    ("mrn_schema_begin_group", ctypes.c_int, [vp, ctypes.c_char_p]),
    ("mrn_schema_end_group", ctypes.c_int, [vp]),
    ("mrn_schema_add_jagged", ctypes.c_int, [vp, ctypes.c_char_p, ctypes.c_int, vp]),
    ("mrn_schema_finalize", ctypes.c_int, [vp]),
    ("mrn_schema_destroy", None, [vp]),
    ("mrn_schema_info_get", ctypes.c_int, [vp, ctypes.POINTER(SchemaInfo)]),
    ("mrn_schema_column", ctypes.c_int, [vp, ctypes.c_int, u32, ctypes.POINTER(ColumnInfo)]),
    ("mrn_schema_aos_layout", ctypes.c_int, [vp, ctypes.POINTER(sz), ctypes.POINTER(sz), sz]),
    ("mrn_required_bytes", ctypes.c_int, [vp, Layout, u64, u64, ctypes.POINTER(sz)]),
    ("mrn_child_pool_bytes", ctypes.c_int, [vp, u64, ctypes.POINTER(sz)]),
    ("mrn_soa_region_offset", ctypes.c_int, [vp, u64, u64, u32, ctypes.POINTER(sz)]),
    ("mrn_region_offset", ctypes.c_int, [vp, Layout, u64, u64, u32, ctypes.POINTER(sz)]),
    ("mrn_aosoa_block_bytes", ctypes.c_int, [vp, u32, ctypes.POINTER(sz)]),
    ("mrn_aosoa_column_offset", ctypes.c_int, [vp, u32, u32, ctypes.POINTER(sz)]),
    ("mrn_convert", ctypes.c_int, [ctypes.POINTER(ViewStruct), ctypes.POINTER(ViewStruct), vp]),
    ("mrn_convert_jagged_noalloc", ctypes.c_int, [ctypes.POINTER(ViewStruct), ctypes.POINTER(ViewStruct), vp]),
    ("mrn_sync", ctypes.c_int, [vp]),
    ("mrn_sync_bits", ctypes.c_int, [vp, ctypes.POINTER(u32)]),
    ("mrn_scratch_release", ctypes.c_int, [ctypes.c_int]),
    ("mrn_jagged_count", ctypes.c_int, [ctypes.POINTER(ViewStruct), ctypes.POINTER(u64), vp]),
    ("mrn_debug_set", ctypes.c_int, [ctypes.c_int, ctypes.c_longlong]),
    ("mrn_transfer_convert", ctypes.c_int, [ctypes.POINTER(ViewStruct), ctypes.POINTER(ViewStruct),
                                            ctypes.POINTER(TransferOpts), vp]),
    ("mrn_batch_create", ctypes.c_int, [ctypes.POINTER(Job), sz, ctypes.c_int, ctypes.POINTER(vp)]),
    ("mrn_batch_launch", ctypes.c_int, [vp, vp]),
    ("mrn_batch_launch_timed", ctypes.c_int, [vp, vp, vp, vp, vp]),
    ("mrn_batch_launch_per_job", ctypes.c_int, [vp, vp]),
    ("mrn_batch_update", ctypes.c_int, [vp, sz, ctypes.POINTER(ViewStruct), ctypes.POINTER(ViewStruct)]),
    ("mrn_batch_destroy", None, [vp]),
    ("mrn_batch_tune", ctypes.c_int, [vp, vp, ctypes.POINTER(BatchTuneResult)]),
    ("mrn_autotune", ctypes.c_int, [vp, Layout, Layout, u64, ctypes.POINTER(TuneResult)]),
    ("mrn_autotune_clear", ctypes.c_int, []),
    ("mrn_server_create", ctypes.c_int, [ctypes.POINTER(ServerOpts), ctypes.POINTER(vp)]),
    ("mrn_server_submit", ctypes.c_int, [vp, ctypes.POINTER(ViewStruct), ctypes.POINTER(ViewStruct),
                                         ctypes.POINTER(u64)]),
    ("mrn_server_poll", ctypes.c_int, [vp, u64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    ("mrn_server_wait", ctypes.c_int, [vp, u64, u64, ctypes.POINTER(ctypes.c_int)]),
    ("mrn_server_wait_latency", ctypes.c_int, [vp, u64, u64, ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(ctypes.c_double)]),
    ("mrn_server_stats_get", ctypes.c_int, [vp, ctypes.POINTER(ServerStats)]),
    ("mrn_server_destroy", None, [vp]),
    ("mrn_memmove", ctypes.c_int, [vp, vp, u64, ctypes.c_int, vp]),
    ("mrn_collection_create", ctypes.c_int, [vp, Layout, ctypes.c_int, ctypes.c_int, u64, u64,
                                             ctypes.POINTER(vp)]),
    ("mrn_collection_destroy", None, [vp]),
    ("mrn_collection_view", ctypes.c_int, [vp, ctypes.POINTER(ViewStruct)]),
    ("mrn_collection_sizes", ctypes.c_int, [vp, ctypes.POINTER(u64), ctypes.POINTER(u64),
                                            ctypes.POINTER(u64), ctypes.POINTER(u64)]),
    ("mrn_collection_reserve", ctypes.c_int, [vp, u64, u64, vp]),
    ("mrn_collection_resize", ctypes.c_int, [vp, u64, vp]),
    ("mrn_collection_clear", ctypes.c_int, [vp, vp]),
    ("mrn_collection_shrink_to_fit", ctypes.c_int, [vp, vp]),
    ("mrn_collection_erase", ctypes.c_int, [vp, u64, u64, vp]),
    ("mrn_collection_insert", ctypes.c_int, [vp, u64, ctypes.POINTER(ViewStruct), vp]),
    ("mrn_collection_assign", ctypes.c_int, [vp, ctypes.POINTER(ViewStruct), vp]),
    ("mrn_collection_set_context", ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp]),
]

_lib = None


def lib():
    """The loaded library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libmrn.so is not built (run paper_2511_04853_b300/build.py); "
                              "there is no fallback path")
        L = ctypes.CDLL(LIB_PATH)
        for name, rt, at in SIGNATURES:
            f = getattr(L, name, None)
            if f is None:
                continue
            f.restype, f.argtypes = rt, at
        _lib = L
    return _lib


class MrnError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__("%s%s" % (status_str(code), (": " + what) if what else ""))


def status_str(code):
    return lib().mrn_status_str(code).decode()


def check(code, what=""):
    if code != OK:
        raise MrnError(code, what)
    return code


_CURRENT_STREAM = []  # torch.cuda.current_stream once CUDA is known to be available


def _stream(stream):
    if stream is None:
        if _CURRENT_STREAM:
            return _CURRENT_STREAM[0]().cuda_stream
        try:
            import torch
            if torch.cuda.is_available():
                _CURRENT_STREAM.append(torch.cuda.current_stream)
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(x):
    """Address of a torch tensor, numpy array or integer."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(type(x))


class Schema:
    """A finalized library schema built from a description list (see
    ``datagen.schemas`` for the format)."""

    def __init__(self, desc):
        L = lib()
        h = vp()
        check(L.mrn_schema_create(ctypes.byref(h)))
        self._h = h
        self.desc = desc
        self._children = []
        try:
            self._add(desc)
            check(L.mrn_schema_finalize(self._h), "finalize")
        except Exception:
            L.mrn_schema_destroy(self._h)
            self._h = None
            raise
        info = SchemaInfo()
        check(L.mrn_schema_info_get(self._h, ctypes.byref(info)))
        self.info = info
        self.ncols = info.n_columns
        self.stride = info.aos_stride
        self.has_jagged = bool(info.has_jagged)
        self.hash = info.hash
        self.columns = [self.column(c) for c in range(self.ncols)]
        self.child_columns = [self.column(c, child=True) for c in range(info.child_columns)]

    def _add(self, desc):
        L = lib()
        for m in desc:
            name = m[0].encode()
            if m[1] == "group":
                check(L.mrn_schema_begin_group(self._h, name))
                self._add(m[2])
                check(L.mrn_schema_end_group(self._h))
            elif m[1] == "jagged":
                child = Schema(m[3])
                self._children.append(child)
                check(L.mrn_schema_add_jagged(self._h, name, DTYPES[m[2]], child._h))
            elif len(m) > 3 and m[3] == "interleaved":
                check(L.mrn_schema_add_field_interleaved(self._h, name, DTYPES[m[1]], int(m[2])), m[0])
            else:
                check(L.mrn_schema_add_field(self._h, name, DTYPES[m[1]], int(m[2])), m[0])

    def column(self, c, child=False):
        ci = ColumnInfo()
        check(lib().mrn_schema_column(self._h, 1 if child else 0, c, ctypes.byref(ci)))
        return {"size": ci.size, "aos_offset": ci.aos_offset, "dtype": ci.dtype,
                "fm_stride": ci.fm_stride, "name": ci.name.decode()}

    def required_bytes(self, kind, n, m=0, block=0):
        out = sz()
        check(lib().mrn_required_bytes(self._h, Layout(KIND.get(kind, kind), block), n, m,
                                       ctypes.byref(out)))
        return out.value

    def child_pool_bytes(self, m):
        out = sz()
        check(lib().mrn_child_pool_bytes(self._h, m, ctypes.byref(out)))
        return out.value

    def required_bytes_nested(self, kind, n, m, m2, block=0):
        out = sz()
        check(lib().mrn_required_bytes_nested(self._h, Layout(KIND.get(kind, kind), block), n, m, m2,
                                              ctypes.byref(out)))
        return out.value

    def grandchild_pool_bytes(self, m2):
        out = sz()
        check(lib().mrn_grandchild_pool_bytes(self._h, m2, ctypes.byref(out)))
        return out.value

    def region_offset_nested(self, kind, n, m, m2, r, block=0):
        out = sz()
        check(lib().mrn_region_offset_nested(self._h, Layout(KIND.get(kind, kind), block), n, m, m2, r,
                                             ctypes.byref(out)))
        return out.value

    def region_offset(self, kind, n, m, r, block=0):
        out = sz()
        check(lib().mrn_region_offset(self._h, Layout(KIND.get(kind, kind), block), n, m, r,
                                      ctypes.byref(out)))
        return out.value

    def soa_region_offset(self, n, m, r):
        out = sz()
        check(lib().mrn_soa_region_offset(self._h, n, m, r, ctypes.byref(out)))
        return out.value

    def aosoa_block_bytes(self, B):
        out = sz()
        check(lib().mrn_aosoa_block_bytes(self._h, B, ctypes.byref(out)))
        return out.value

    def aosoa_column_offset(self, B, c):
        out = sz()
        check(lib().mrn_aosoa_column_offset(self._h, B, c, ctypes.byref(out)))
        return out.value

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.mrn_schema_destroy(self._h)
            self._h = None


class View:
    """A ``mrn_view`` over caller-owned buffers (torch tensors, numpy arrays
    or raw addresses).  Keeps the buffer objects alive."""

    def __init__(self, schema, kind, n, block=0, base=None, columns=None, offsets=None,
                 child_columns=None, child_pool=None, m=0, mem="device", device=None,
                 offset_base=0, m2=0, grandchild_pool=None):
        self.schema = schema
        self._keep = [base, columns, offsets, child_columns, child_pool, grandchild_pool]
        if device is None:
            device = 0
            if hasattr(base, "data_ptr") and getattr(base, "is_cuda", False):
                device = base.device.index
        cols_arr = None
        if columns is not None:
            cols_arr = (vp * len(columns))(*[_ptr(c) for c in columns])
        ccols_arr = None
        if child_columns is not None:
            ccols_arr = (vp * len(child_columns))(*[_ptr(c) for c in child_columns])
        self._arrays = [cols_arr, ccols_arr]
        self.s = ViewStruct(
            schema._h, Layout(KIND.get(kind, kind), block), MEM.get(mem, mem), device, n, m,
            _ptr(base), ctypes.cast(cols_arr, vp) if cols_arr is not None else None,
            _ptr(offsets), ctypes.cast(ccols_arr, vp) if ccols_arr is not None else None,
            _ptr(child_pool), offset_base, m2, _ptr(grandchild_pool))

    @property
    def ref(self):
        return ctypes.byref(self.s)


def convert(src, dst, stream=None):
    rc = _LIB_CONVERT[0](src.ref, dst.ref, _stream(stream)) if _LIB_CONVERT else _first_convert(src, dst, stream)
    if rc != OK:
        raise MrnError(rc, "mrn_convert")


_LIB_CONVERT = []


def _first_convert(src, dst, stream):
    _LIB_CONVERT.append(lib().mrn_convert)
    return _LIB_CONVERT[0](src.ref, dst.ref, _stream(stream))


def convert_status(src, dst, stream=None):
    return lib().mrn_convert(src.ref, dst.ref, _stream(stream))


def sync(stream=None):
    """Waits for the stream; returns the first device-recorded status."""
    return lib().mrn_sync(_stream(stream))


def scratch_release(device=0):
    """Returns the library's unused scratch memory on `device`."""
    check(lib().mrn_scratch_release(device))


def sync_bits(stream=None):
    b = u32()
    check(lib().mrn_sync_bits(_stream(stream), ctypes.byref(b)))
    return b.value


def jagged_count(src, stream=None):
    m = u64()
    check(lib().mrn_jagged_count(src.ref, ctypes.byref(m), _stream(stream)))
    return m.value


def debug_set(key, value):
    check(lib().mrn_debug_set(key, value))


TRANSFER_ZERO_COPY = 1


def transfer_convert(src, dst, chunk_bytes=0, n_slots=0, stream=None, zero_copy=False):
    opts = TransferOpts(chunk_bytes, n_slots, TRANSFER_ZERO_COPY if zero_copy else 0)
    check(lib().mrn_transfer_convert(src.ref, dst.ref, ctypes.byref(opts), _stream(stream)),
          "mrn_transfer_convert")


class Batch:
    """Many conversions in one persistent launch (``mrn_batch_*``)."""

    def __init__(self, pairs, use_graph=True):
        self._pairs = list(pairs)
        jobs = (Job * len(self._pairs))()
        for i, (s, d) in enumerate(self._pairs):
            jobs[i].src = ctypes.pointer(s.s)
            jobs[i].dst = ctypes.pointer(d.s)
        h = vp()
        check(lib().mrn_batch_create(jobs, len(self._pairs), 1 if use_graph else 0,
                                     ctypes.byref(h)), "mrn_batch_create")
        self._h = h

    def launch(self, stream=None):
        check(lib().mrn_batch_launch(self._h, _stream(stream)), "mrn_batch_launch")

    def launch_timed(self, ev_begin, ev_mid, ev_end, stream=None):
        """``mrn_batch_launch_timed``: the events (torch.cuda.Event with
        timing) are recorded before the batch, after the scratch reset and
        the fused jagged launch, and after the persistent launches and the
        fall-back pass."""
        evs = []
        for e in (ev_begin, ev_mid, ev_end):
            if not e.cuda_event:  # torch creates an event at its first record
                e.record()
            evs.append(vp(e.cuda_event))
        check(lib().mrn_batch_launch_timed(self._h, _stream(stream), *evs), "mrn_batch_launch_timed")

    def launch_per_job(self, stream=None):
        check(lib().mrn_batch_launch_per_job(self._h, _stream(stream)), "per-job")

    def tune(self, stream=None):
        """Autotunes this batch's launch shape on its own jobs (the trial
        launches write the destinations)."""
        r = BatchTuneResult()
        check(lib().mrn_batch_tune(self._h, _stream(stream), ctypes.byref(r)), "mrn_batch_tune")
        return {"max_chunk": r.max_chunk, "ctas_per_sm": r.ctas_per_sm, "ms": r.ms, "default_ms": r.default_ms,
                "worst_ms": r.worst_ms, "candidates": r.candidates}

    def update(self, j, src, dst):
        self._pairs[j] = (src, dst)
        check(lib().mrn_batch_update(self._h, j, src.ref, dst.ref), "mrn_batch_update")

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.mrn_batch_destroy(self._h)
            self._h = None


def autotune(schema, src_kind, dst_kind, n_hint, src_block=0, dst_block=0):
    r = TuneResult()
    check(lib().mrn_autotune(schema._h, Layout(KIND.get(src_kind, src_kind), src_block),
                             Layout(KIND.get(dst_kind, dst_kind), dst_block), n_hint,
                             ctypes.byref(r)), "mrn_autotune")
    return {"threads": r.threads, "ctas_per_sm": r.ctas_per_sm, "tile_records": r.tile_records,
            "staged": bool(r.staged), "gbps": r.gbps, "default_gbps": r.default_gbps}


def autotune_clear():
    check(lib().mrn_autotune_clear())


class Server:
    """Continuous-batching conversion server (``mrn_server_*``)."""

    def __init__(self, hbm_budget_bytes, max_slots=8, chunk_bytes=0):
        opts = ServerOpts(hbm_budget_bytes, max_slots, 0, chunk_bytes)
        h = vp()
        check(lib().mrn_server_create(ctypes.byref(opts), ctypes.byref(h)), "mrn_server_create")
        self._h = h
        self._live = {}

    def submit(self, src, dst):
        t = u64()
        rc = lib().mrn_server_submit(self._h, src.ref, dst.ref, ctypes.byref(t))
        if rc != OK:
            return rc, None
        self._live[t.value] = (src, dst)
        return OK, t.value

    def poll(self, ticket):
        done, st = ctypes.c_int(), ctypes.c_int()
        check(lib().mrn_server_poll(self._h, ticket, ctypes.byref(done), ctypes.byref(st)))
        if done.value:
            self._live.pop(ticket, None)
        return bool(done.value), st.value

    def wait(self, ticket, timeout_s=60.0):
        st = ctypes.c_int()
        rc = lib().mrn_server_wait(self._h, ticket, int(timeout_s * 1e9), ctypes.byref(st))
        if rc == OK:
            self._live.pop(ticket, None)
            return st.value
        return rc

    def wait_latency(self, ticket, timeout_s=60.0):
        """Waits for the request; returns (status, latency in ms)."""
        st, lat = ctypes.c_int(), ctypes.c_double()
        rc = lib().mrn_server_wait_latency(self._h, ticket, int(timeout_s * 1e9), ctypes.byref(st),
                                           ctypes.byref(lat))
        if rc == OK:
            self._live.pop(ticket, None)
            return st.value, lat.value
        return rc, None

    def stats(self):
        s = ServerStats()
        check(lib().mrn_server_stats_get(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.mrn_server_destroy(self._h)
            self._h = None
            self._live.clear()

    def __del__(self):
        self.close()


def memmove(dst, src, nbytes, mem="device", stream=None):
    """Moves nbytes from src to dst (addresses, tensors or arrays) inside one
    memory context; the ranges may overlap."""
    check(lib().mrn_memmove(_ptr(dst), _ptr(src), nbytes, MEM.get(mem, mem), _stream(stream)),
          "mrn_memmove")


class _CollectionView:
    """The ``mrn_view`` of a collection's current contents (pointer arrays
    owned by the collection: valid until it reallocates)."""

    def __init__(self, schema, s):
        self.schema = schema
        self.s = s

    @property
    def ref(self):
        return ctypes.byref(self.s)


class Collection:
    """A library-owned collection (``mrn_collection``): a schema, a layout
    and a memory context ("device", "pinned" or "host")."""

    def __init__(self, schema, kind, capacity=0, child_capacity=0, block=0, mem="device", device=0):
        self.schema = schema
        h = vp()
        check(lib().mrn_collection_create(schema._h, Layout(KIND.get(kind, kind), block), MEM.get(mem, mem),
                                          device, capacity, child_capacity, ctypes.byref(h)),
              "mrn_collection_create")
        self._h = h

    def view(self):
        v = ViewStruct()
        check(lib().mrn_collection_view(self._h, ctypes.byref(v)), "mrn_collection_view")
        return _CollectionView(self.schema, v)

    def sizes(self):
        """(n, m, capacity, child_capacity)"""
        out = [u64(), u64(), u64(), u64()]
        check(lib().mrn_collection_sizes(self._h, *[ctypes.byref(x) for x in out]), "mrn_collection_sizes")
        return tuple(int(x.value) for x in out)

    def reserve(self, capacity, child_capacity=0, stream=None):
        check(lib().mrn_collection_reserve(self._h, capacity, child_capacity, _stream(stream)),
              "mrn_collection_reserve")

    def resize(self, n, stream=None):
        check(lib().mrn_collection_resize(self._h, n, _stream(stream)), "mrn_collection_resize")

    def clear(self, stream=None):
        check(lib().mrn_collection_clear(self._h, _stream(stream)), "mrn_collection_clear")

    def shrink_to_fit(self, stream=None):
        check(lib().mrn_collection_shrink_to_fit(self._h, _stream(stream)), "mrn_collection_shrink_to_fit")

    def erase(self, first, count, stream=None):
        check(lib().mrn_collection_erase(self._h, first, count, _stream(stream)), "mrn_collection_erase")

    def insert(self, pos, src, stream=None):
        check(lib().mrn_collection_insert(self._h, pos, src.ref, _stream(stream)), "mrn_collection_insert")

    def assign(self, src, stream=None):
        check(lib().mrn_collection_assign(self._h, src.ref, _stream(stream)), "mrn_collection_assign")

    def set_context(self, mem, device=0, stream=None):
        check(lib().mrn_collection_set_context(self._h, MEM.get(mem, mem), device, _stream(stream)),
              "mrn_collection_set_context")

    def close(self):
        if getattr(self, "_h", None):
            lib().mrn_collection_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
