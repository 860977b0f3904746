"""Shared helpers of the nested jagged tests: re-laying child runs in a pool."""
import numpy as np


def shuffle_runs(recs, count, stride, len_off, begin_off, pool, rsize, order, gap):
    """Re-lays the runs that `count` records (stride bytes each, with a
    {u32 length @len_off, u64 begin @begin_off} descriptor) own in `pool`
    (rsize-byte records): record order[k]'s run goes k-th, `gap` empty slots
    before each; the begins are rewritten.  Returns the new pool."""
    lens = [int(recs[i * stride + len_off: i * stride + len_off + 4].view("<u4")[0]) for i in range(count)]
    begs = [int(recs[i * stride + begin_off: i * stride + begin_off + 8].view("<u8")[0]) for i in range(count)]
    out = np.zeros(max(1, (sum(lens) + gap * count) * rsize), np.uint8)
    cur = 0
    for i in order:
        i = int(i)
        cur += gap
        out[cur * rsize:(cur + lens[i]) * rsize] = pool[begs[i] * rsize:(begs[i] + lens[i]) * rsize]
        recs[i * stride + begin_off: i * stride + begin_off + 8] = np.array([cur], "<u8").view(np.uint8)
        cur += lens[i]
    return out


def shuffled_nested(o, aos, seed, gap=1):
    """The canonical nested AoS side `aos` (oracle side of schema `o`) with
    both pools re-laid: grandchild runs, then child runs, in seeded random
    orders with `gap` free slots before each run.  Returns (records,
    child pool, grandchild pool, child slots, grandchild slots)."""
    m, m2 = aos.m, aos.m2
    cs, gs = o.child.stride, o.child.child.stride
    rng = np.random.default_rng(seed)
    kids = aos.pool[: max(1, m * cs)].copy()
    gpool = shuffle_runs(kids, m, cs, o.child.len_off, o.child.begin_off, aos.gpool, gs, rng.permutation(m), gap)
    recs = aos.base.copy()
    pool = shuffle_runs(recs, aos.n, o.stride, o.len_off, o.begin_off, kids, cs, rng.permutation(aos.n), gap)
    return recs, pool, gpool, (pool.size // cs) if m else 0, (gpool.size // gs) if m2 else 0
