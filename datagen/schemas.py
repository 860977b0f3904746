"""Record schemas of the workloads, as plain data.

A schema is a list of members. Each member is one of

* ``(name, dtype, extent)``            a per-item property (extent 1) or a
                                       fixed-extent array property (Sec. V,
                                       "per-item property", "array property"),
                                       stored field-major as E separate columns
* ``(name, dtype, extent, "interleaved")``
                                       an array property stored field-major as
                                       one N x E array (the property's other
                                       interface in Sec. V)
* ``(name, "group", [members])``       a sub-group property (Sec. V)
* ``(name, "jagged", offset_dtype, [members])``
                                       a jagged vector property (Sec. V); the
                                       offset dtype is the prefix-sum type

``dtype`` is one of the names in :data:`DTYPE_SIZES`.  This module holds no
layout arithmetic: it only names fields and their element types.  Both the
oracle and the CUDA library build their own layouts from these lists.
"""

DTYPE_SIZES = {
    "u8": 1, "i8": 1, "bool": 1,
    "u16": 2, "i16": 2,
    "u32": 4, "i32": 4, "f32": 4,
    "u64": 8, "i64": 8, "f64": 8,
}

# numpy storage type of each dtype; bool is stored as a raw byte so that
# byte values other than 0/1 survive every conversion unchanged.
NUMPY_TYPES = {
    "u8": "<u1", "i8": "<i1", "bool": "<u1",
    "u16": "<u2", "i16": "<i2",
    "u32": "<u4", "i32": "<i4", "f32": "<f4",
    "u64": "<u8", "i64": "<i8", "f64": "<f8",
}

# 10,000-record point collection: x, y, z, id, key, flag.
POINTS = [
    ("x", "f32", 1), ("y", "f32", 1), ("z", "f32", 1),
    ("id", "i32", 1), ("key", "u64", 1), ("flag", "u8", 1),
]

# Calorimeter-cell-like collection (200,000 records).
CELLS = [
    ("energy", "f32", 1), ("time", "f32", 1), ("eta", "f32", 1),
    ("phi", "f32", 1), ("cell_id", "u32", 1), ("gain", "u16", 1),
    ("quality", "u16", 1),
]

# Jagged collection: parents {pt, eta, label} with a child array of
# {index, weight}, uint32 prefix sums.
TRACKS = [
    ("pt", "f32", 1), ("eta", "f32", 1), ("label", "i32", 1),
    ("hits", "jagged", "u32", [("index", "u32", 1), ("weight", "f32", 1)]),
]

# Jagged with a nested jagged member: every hit of a track holds a list of
# {time, adc} samples (Poisson(3) per hit, clipped at 32), uint32 prefix
# sums at both levels.
TRACKS_NESTED = [
    ("pt", "f32", 1), ("eta", "f32", 1), ("label", "i32", 1),
    ("hits", "jagged", "u32", [("index", "u32", 1), ("weight", "f32", 1),
                                ("samples", "jagged", "u32", [("t", "u16", 1), ("adc", "u16", 1)])]),
]

# The motivating example's Sensor (Listing 1 / Listing 3): an enum stored in
# one byte, a sub-group of calibration constants.
SENSOR = [
    ("type", "u8", 1), ("counts", "u64", 1), ("energy", "f32", 1),
    ("calibration_data", "group", [
        ("noisy", "bool", 1), ("parameter_A", "f32", 1),
        ("parameter_B", "f32", 1), ("noise_A", "f32", 1),
        ("noise_B", "f32", 1),
    ]),
]

# The motivating example's Particle (Listing 2 / Listing 3) with
# SensorType::Num = 4: arrays tracked per sensor type and a jagged list of
# sensor ids.
SENSOR_TYPES = 4
PARTICLE = [
    ("energy", "f32", 1), ("x", "f32", 1), ("y", "f32", 1),
    ("origin", "u64", 1),
    ("sensors", "jagged", "u32", [("id", "u64", 1)]),
    ("x_variance", "f32", 1), ("y_variance", "f32", 1),
    ("significance", "f32", SENSOR_TYPES),
    ("E_contribution", "f32", SENSOR_TYPES),
    ("noisy_count", "u8", SENSOR_TYPES),
]

# The points collection with its position as one interleaved f32[3] array
# property (one N x 3 array field-major): the same AoS record as POINTS.
POINTS_INTERLEAVED = [
    ("pos", "f32", 3, "interleaved"),
    ("id", "i32", 1), ("key", "u64", 1), ("flag", "u8", 1),
]

WORKLOAD_SCHEMAS = {"points": POINTS, "cells": CELLS, "tracks": TRACKS}
NESTED_SCHEMAS = {"tracks_nested": TRACKS_NESTED}
INTERLEAVED_SCHEMAS = {"points_interleaved": POINTS_INTERLEAVED}


def leaves(schema, prefix=""):
    """Depth-first list of ``(path, dtype, extent)`` for the data members of a
    schema (groups are descended into, the jagged member is skipped)."""
    out = []
    for m in schema:
        if m[1] == "group":
            out += leaves(m[2], prefix + m[0] + ".")
        elif m[1] == "jagged":
            continue
        else:
            out.append((prefix + m[0], m[1], m[2]))
    return out


def jagged_member(schema):
    """Return ``(name, offset_dtype, child_schema)`` of the jagged member or
    None.  Searches groups too."""
    for m in schema:
        if m[1] == "jagged":
            return m[0], m[2], m[3]
        if m[1] == "group":
            j = jagged_member(m[2])
            if j is not None:
                return j
    return None
