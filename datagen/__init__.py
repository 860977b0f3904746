"""Seeded synthetic workload inputs, shared by the tests, the oracle's
drivers and the benchmark.  Holds no layout or conversion arithmetic."""
from .schemas import (DTYPE_SIZES, NUMPY_TYPES, POINTS, CELLS, TRACKS,  # noqa: F401
                      SENSOR, PARTICLE, WORKLOAD_SCHEMAS, TRACKS_NESTED, NESTED_SCHEMAS,
                      POINTS_INTERLEAVED, INTERLEAVED_SCHEMAS, leaves, jagged_member)
from .generate import (workload, random_columns, jagged_random,  # noqa: F401
                       raw_bits, pool_permutation)
