"""Size-changing operations on a collection's values — TEST INFRASTRUCTURE
ONLY (the same import rule as the rest of ``oracle``).

The plain definitions of the layout holder's size-changing operations
(Sec. VI-B: resize, clear, insert, erase), written on the logical contents
of a collection rather than on any layout: the generator's value dict
``{"n", "columns", and for a jagged schema "lengths", "children", "m"}``
(per-member arrays, one row per object; the children of object i are rows
``sum(lengths[:i]) ..`` of the child arrays, in object order).  Laying the
result out is ``oracle.pack``'s job.

* erase(first, count): the objects [first, first + count) and their
  children disappear; the rest keep their order.
* insert(pos, other): the objects of ``other`` (and their children) come
  before object ``pos``.
* resize(n): the first n objects when shrinking; all-zero objects with no
  children appended when growing (the value-initialised objects of a
  vector-like container).
"""
import numpy as np


def _copy(d):
    out = dict(d)
    out["columns"] = [np.asarray(c).copy() for c in d["columns"]]
    if "lengths" in d:
        out["lengths"] = np.asarray(d["lengths"]).copy()
        out["children"] = [np.asarray(c).copy() for c in d["children"]]
    return out


def _child_start(d, i):
    """Index of the first child row of object i."""
    return int(np.asarray(d["lengths"][:i], dtype=np.uint64).sum())


def erase(d, first, count):
    n = d["n"]
    assert 0 <= first <= n and 0 <= count <= n - first
    out = _copy(d)
    keep = np.r_[0:first, first + count:n]
    out["columns"] = [c[keep] for c in d["columns"]]
    out["n"] = n - count
    if "lengths" in d:
        a, b = _child_start(d, first), _child_start(d, first + count)
        m = d["m"]
        kkeep = np.r_[0:a, b:m]
        out["lengths"] = np.asarray(d["lengths"])[keep]
        out["children"] = [c[kkeep] for c in d["children"]]
        out["m"] = m - (b - a)
    return out


def insert(d, pos, other):
    n = d["n"]
    assert 0 <= pos <= n
    out = _copy(d)
    out["columns"] = [np.concatenate([c[:pos], o, c[pos:]]) for c, o in zip(d["columns"], other["columns"])]
    out["n"] = n + other["n"]
    if "lengths" in d:
        a = _child_start(d, pos)
        out["lengths"] = np.concatenate([d["lengths"][:pos], other["lengths"], d["lengths"][pos:]]).astype(
            np.asarray(d["lengths"]).dtype)
        out["children"] = [np.concatenate([c[:a], o, c[a:]]) for c, o in zip(d["children"], other["children"])]
        out["m"] = d["m"] + other["m"]
    return out


def resize(d, n):
    if n <= d["n"]:
        return erase(d, n, d["n"] - n)
    k = n - d["n"]
    out = _copy(d)
    out["columns"] = [np.concatenate([c, np.zeros((k,) + c.shape[1:], c.dtype)]) for c in d["columns"]]
    out["n"] = n
    if "lengths" in d:
        ln = np.asarray(d["lengths"])
        out["lengths"] = np.concatenate([ln, np.zeros(k, ln.dtype)])
    return out


def take(d, first, count):
    """The objects [first, first + count) as a collection of their own."""
    return erase(erase(d, first + count, d["n"] - first - count), 0, first)
