"""Record-range sharding of one collection across the ranks of a process
group (one GPU per rank; this library runs replicas only, so nothing here
launches device work).

Records are independent, so a collection splits into contiguous record
ranges, one per rank, each converted on its rank's GPU with the ordinary
calls.  Every range starts on a multiple of an alignment, the least common
multiple of the AoSoA blocks B of both sides and of the caller's tile, so
that each rank's AoSoA blocks are whole.

The only dependency across ranks is the jagged prefix sum (Sec. V, jagged
vector property: the offsets are the prefix sum of the sizes).  A rank's
offsets start at the number of children of all earlier ranks.
``child_base`` obtains that number with one all-gather of a single 64-bit
count per rank and an exclusive scan on the host; the rank then converts
with ``offset_base`` set to it (``mrn_view.offset_base``), which makes its
offsets global.  Concatenating the ranks' offset columns (each rank's last
entry dropped, except the last rank's) and their child columns gives the
whole collection's.
"""
import math


def alignment(*blocks):
    """Least common multiple of the given record granules (AoSoA block
    sizes, tile sizes); zeros and Nones are ignored."""
    a = 1
    for b in blocks:
        if b:
            a = a * int(b) // math.gcd(a, int(b))
    return a


def shard_range(n, rank, world, align=1):
    """Records [lo, hi) of rank ``rank`` of ``world``: contiguous, disjoint,
    covering [0, n), every lo a multiple of ``align``, and the counts of
    align-sized units balanced to within one unit."""
    if world < 1 or not 0 <= rank < world or align < 1 or n < 0:
        raise ValueError("bad shard request")
    units = -(-n // align)
    lo = min(n, units * rank // world * align)
    hi = min(n, units * (rank + 1) // world * align)
    return lo, hi


def exclusive_bases(counts):
    """Exclusive prefix sums of per-rank child counts and their total."""
    out, run = [], 0
    for c in counts:
        out.append(run)
        run += int(c)
    return out, run


def child_base(local_children, group=None, device=None):
    """This rank's child base (children of all earlier ranks) and the total,
    from one all-gather of one 64-bit count per rank over ``group``
    (torch.distributed; ``device`` is where the exchanged tensor lives, for
    example ``cuda`` under NCCL, the CPU under gloo)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    mine = torch.tensor([int(local_children)], dtype=torch.int64, device=device)
    parts = [torch.zeros(1, dtype=torch.int64, device=device) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    bases, total = exclusive_bases([int(p.item()) for p in parts])
    return bases[rank], total
