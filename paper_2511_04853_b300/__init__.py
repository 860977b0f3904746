"""B300-native (sm_103a) schema-driven layout conversion.

Converts collections of records between array-of-structures, structure-of-
arrays, blocked (AoSoA) and jagged (offsets + values) layouts on the GPU, fused
with host<->device transfer, following "Marionette: Data Structure
Description and Management for Heterogeneous Computing" (arXiv 2511.04853).
The work happens in ``libmrn.so`` (C ABI in ``include/mrn.h``); this package
is its ctypes binding plus host-side helpers.
"""
from .mrn import (  # noqa: F401
    lib, Schema, View, convert, convert_status, sync, sync_bits, jagged_count,
    transfer_convert, Batch, autotune, autotune_clear, Server, MrnError,
    memmove, Collection, scratch_release,
    status_str, debug_set, AOS, SOA, AOSOA, OK, EINVAL, ESIZE, EALIGN,
    EOVERFLOW, ENOMEM, ETIMEOUT, ECUDA, EBUSY, ENOTFOUND, EUNSUPPORTED)
