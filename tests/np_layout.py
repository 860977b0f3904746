"""numpy's own C-layout machinery, used to pin the oracle.

``numpy.dtype(..., align=True)`` lays out structured types with the C
compiler's natural-alignment rules (nested structs aligned to their widest
member, trailing padding), so it is an implementation of the AoS and
AoSoA-block rules that shares nothing with the oracle.
"""
import numpy as np

from datagen import NUMPY_TYPES, leaves


def struct_dtype(desc):
    """C struct of a schema: groups are nested structs, an array property is
    a subarray, the jagged member is ``{uint32 length; uint64 begin}`` as two
    members at its position."""
    fields = []
    for m in desc:
        if m[1] == "group":
            fields.append((m[0], struct_dtype(m[2])))
        elif m[1] == "jagged":
            fields.append((m[0] + "_length", "<u4"))
            fields.append((m[0] + "_begin", "<u8"))
        elif m[2] == 1:
            fields.append((m[0], NUMPY_TYPES[m[1]]))
        else:
            fields.append((m[0], NUMPY_TYPES[m[1]], (m[2],)))
    return np.dtype(fields, align=True)


def leaf_paths(desc):
    return [(p.split("."), dt, e) for p, dt, e in leaves(desc)]


def get_leaf(arr, path):
    for p in path:
        arr = arr[p]
    return arr


def flat_column_types(desc):
    """numpy type of each flattened column."""
    out = []
    for _, dt, e in leaves(desc):
        out += [NUMPY_TYPES[dt]] * e
    return out


def aos_from_values(desc, values, n):
    """Zero-filled aligned structured array with the leaves filled."""
    dt = struct_dtype(desc)
    arr = np.zeros(n, dt)
    for (path, _, _), v in zip(leaf_paths(desc), values):
        tgt = arr
        for p in path[:-1]:
            tgt = tgt[p]
        tgt[path[-1]] = v
    return arr


def aos_columns(desc, aos_bytes, n):
    """Flattened column arrays read from AoS bytes through numpy."""
    dt = struct_dtype(desc)
    arr = np.frombuffer(aos_bytes[: n * dt.itemsize].tobytes(), dt, count=n)
    cols = []
    for path, _, e in leaf_paths(desc):
        v = get_leaf(arr, path)
        if e == 1:
            cols.append(np.ascontiguousarray(v))
        else:
            for k in range(e):
                cols.append(np.ascontiguousarray(v[:, k]))
    return cols


def block_dtype(desc, B):
    """AoSoA block as the C struct of B-element column arrays."""
    return np.dtype([("c%d" % k, t, (B,))
                     for k, t in enumerate(flat_column_types(desc))], align=True)


def aosoa_columns(desc, base, n, B):
    dt = block_dtype(desc, B)
    nb = (n + B - 1) // B
    blocks = np.frombuffer(base[: nb * dt.itemsize].tobytes(), dt, count=nb)
    return [np.ascontiguousarray(blocks["c%d" % k].reshape(-1)[:n])
            for k in range(len(dt.names))], blocks


def fill_block_column(blocks, c, col, n):
    """Writes column ``c`` (n values) into an array of AoSoA block structs."""
    fld = blocks["c%d" % c]
    full = np.zeros(fld.size, fld.dtype)
    full[:n] = np.asarray(col).view(fld.dtype)
    fld[...] = full.reshape(fld.shape)


def leaf_kinds(desc):
    """(dtype, extent, interleaved) of every data leaf, depth first."""
    out = []
    for m in desc:
        if m[1] == "group":
            out += leaf_kinds(m[2])
        elif m[1] == "jagged":
            continue
        else:
            out.append((m[1], m[2], len(m) > 3 and m[3] == "interleaved"))
    return out


def storage_block_dtype(desc, B):
    """AoSoA block as a C struct with one member per field-major storage
    column: a B-element array per separately stored column, and a B x E
    array for an interleaved array property (record r's row r)."""
    fields, k = [], 0
    for dt, e, inter in leaf_kinds(desc):
        if inter:
            fields.append(("s%d" % k, NUMPY_TYPES[dt], (B, e)))
            k += 1
        else:
            for _ in range(e):
                fields.append(("s%d" % k, NUMPY_TYPES[dt], (B,)))
                k += 1
    return np.dtype(fields, align=True)


def storage_values(desc, values):
    """Each storage column's values as a C-contiguous array: one per
    separately stored column, the (n, E) rows of an interleaved array."""
    out = []
    for (dt, e, inter), v in zip(leaf_kinds(desc), values):
        v = np.asarray(v)
        if inter or v.ndim == 1:
            out.append(np.ascontiguousarray(v))
        else:
            out += [np.ascontiguousarray(v[:, k]) for k in range(e)]
    return out
