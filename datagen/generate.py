"""Seeded synthetic inputs shaped like the paper's workloads.

Every generator returns *logical values*: one numpy array per data leaf of
the schema (shape ``(n,)`` for a scalar, ``(n, extent)`` for an array
property), and for a jagged schema the per-object vector lengths plus the
child leaves in canonical (parent-major) order.  Nothing here places bytes
in a layout; callers hand these arrays to the oracle or to the library.

Seeds use numpy's PCG64 (``default_rng``).  The paper's ATLAS event data is
not available; these distributions stand in for it.
"""
import numpy as np

from .schemas import NUMPY_TYPES, leaves, jagged_member


def raw_bits(rng, dtype, shape):
    """Uniform random bytes viewed as ``dtype`` (NaN payloads, -0.0,
    denormals and bool bytes other than 0/1 all occur)."""
    nt = np.dtype(NUMPY_TYPES[dtype])
    count = int(np.prod(shape, dtype=np.int64)) if len(shape) else 1
    b = rng.integers(0, 256, size=count * nt.itemsize, dtype=np.uint8)
    return b.view(nt).reshape(shape)


def _leaf_shape(n, extent):
    return (n,) if extent == 1 else (n, extent)


def random_columns(schema, n, seed, raw=True):
    """Values for every data leaf of an arbitrary schema: raw random bits."""
    rng = np.random.default_rng(seed)
    cols = [raw_bits(rng, dt, _leaf_shape(n, e)) for _, dt, e in leaves(schema)]
    return {"columns": cols, "n": n}


def _points(n, rng):
    f = lambda: rng.uniform(-1.0, 1.0, n).astype(np.float32)  # noqa: E731
    x, y, z = f(), f(), f()
    ident = rng.integers(-2**31, 2**31, n, dtype=np.int64).astype(np.int32)
    key = rng.integers(0, 2**64, n, dtype=np.uint64)
    flag = rng.integers(0, 256, n, dtype=np.uint8)
    return [x, y, z, ident, key, flag]


def _cells(n, rng):
    energy = rng.exponential(0.5, n).astype(np.float32)
    time = rng.normal(0.0, 5.0, n).astype(np.float32)
    eta = rng.uniform(-4.9, 4.9, n).astype(np.float32)
    phi = rng.uniform(-np.pi, np.pi, n).astype(np.float32)
    cell_id = rng.permutation(n).astype(np.uint32)
    gain = rng.integers(0, 4, n, dtype=np.uint16)
    quality = rng.integers(0, 65536, n, dtype=np.uint16)
    return [energy, time, eta, phi, cell_id, gain, quality]


def _tracks(n, rng, mean_len=20.0, max_len=256):
    pt = rng.exponential(10.0, n).astype(np.float32)
    eta = rng.uniform(-2.5, 2.5, n).astype(np.float32)
    label = rng.integers(0, 10, n, dtype=np.int32)
    lengths = np.minimum(rng.poisson(mean_len, n), max_len).astype(np.uint32)
    m = int(lengths.sum(dtype=np.uint64))
    index = rng.integers(0, 2**32, m, dtype=np.uint64).astype(np.uint32)
    weight = rng.uniform(0.0, 1.0, m).astype(np.float32)
    return [pt, eta, label], lengths, [index, weight]


def workload(name, n, seed, raw=False, mean_len=20.0, max_len=256):
    """Inputs for one of the named workloads (``points``, ``cells``,
    ``tracks``).  ``raw=True`` replaces every value by raw random bits with
    the same shapes (jagged lengths keep their distribution)."""
    rng = np.random.default_rng(seed)
    if name == "points":
        cols = _points(n, rng)
        out = {"columns": cols, "n": n}
    elif name == "cells":
        cols = _cells(n, rng)
        out = {"columns": cols, "n": n}
    elif name == "tracks":
        cols, lengths, kids = _tracks(n, rng, mean_len, max_len)
        out = {"columns": cols, "n": n, "lengths": lengths,
               "children": kids, "m": int(lengths.sum(dtype=np.uint64))}
    elif name == "tracks_nested":
        cols, lengths, kids = _tracks(n, rng, mean_len, max_len)
        m = int(lengths.sum(dtype=np.uint64))
        l1 = np.minimum(rng.poisson(3.0, m), 32).astype(np.uint32)
        m2 = int(l1.sum(dtype=np.uint64))
        t = rng.integers(0, 65536, m2, dtype=np.uint16)
        adc = rng.integers(0, 4096, m2, dtype=np.uint16)
        out = {"columns": cols, "n": n, "lengths": lengths, "children": kids, "m": m,
               "child_lengths": l1, "grandchildren": [t, adc], "m2": m2}
    else:
        raise ValueError(name)
    if raw:
        rr = np.random.default_rng(seed + 1_000_003)
        out["columns"] = [raw_bits(rr, _np_to_name(c.dtype), c.shape)
                          for c in out["columns"]]
        for key in ("children", "grandchildren"):
            if key in out:
                out[key] = [raw_bits(rr, _np_to_name(c.dtype), c.shape) for c in out[key]]
    return out


def jagged_random(schema, n, seed, mean_len=3.0, max_len=16):
    """Values for an arbitrary jagged schema: raw-bit leaves, Poisson
    lengths clipped to ``max_len``."""
    rng = np.random.default_rng(seed)
    cols = [raw_bits(rng, dt, _leaf_shape(n, e)) for _, dt, e in leaves(schema)]
    _, _, child = jagged_member(schema)
    lengths = np.minimum(rng.poisson(mean_len, n), max_len).astype(np.uint32)
    m = int(lengths.sum(dtype=np.uint64))
    kids = [raw_bits(rng, dt, _leaf_shape(m, e)) for _, dt, e in leaves(child)]
    out = {"columns": cols, "n": n, "lengths": lengths, "children": kids, "m": m}
    if jagged_member(child) is not None:
        # a nested jagged member: lengths per child, then the grandchildren
        _, _, grand = jagged_member(child)
        l1 = np.minimum(rng.poisson(mean_len, m), max_len).astype(np.uint32)
        m2 = int(l1.sum(dtype=np.uint64))
        out.update(child_lengths=l1, m2=m2,
                   grandchildren=[raw_bits(rng, dt, _leaf_shape(m2, e)) for _, dt, e in leaves(grand)])
    return out


def pool_permutation(m, seed):
    """A seeded shuffle of child-pool slots (pool order is arbitrary on the
    array-of-structures side)."""
    return np.random.default_rng(seed).permutation(m).astype(np.uint64)


_NAMES = {np.dtype(v).str: k for k, v in NUMPY_TYPES.items() if k != "bool"}


def _np_to_name(dt):
    return _NAMES[np.dtype(dt).str]
