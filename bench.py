"""Benchmark of the layout-conversion hot path on one B300 (or N replicas).

Step: one pass over a batch of R calorimeter-cell collections (200,000
records of {f32 energy, time, eta, phi; u32 cell_id; u16 gain, quality},
24-byte AoS records), each converted AoS -> SoA, SoA -> AoSoA(32) and
AoSoA(32) -> AoS (three independent conversions per collection, each
reading its own resident input), all 3R conversions in ONE persistent kernel
launch replayed from a CUDA graph.  Inputs are resident in HBM; the batch
(R * 6 buffers of 4.8 MB) is larger than the 126 MB L2, so every step
streams from HBM.

value         algorithmic bytes (read + write of every conversion) / step time
e2e           the same bytes through the C ABI with pinned HOST buffers: per
              collection host AoS -> device SoA (transfer-and-convert),
              SoA -> AoSoA(32) on the device, device AoSoA(32) -> host AoS
roofline      the persistent kernel against the measured HBM copy bandwidth
cpu_baseline  the CPU oracle (plain C, one thread) on a bounded sample
batched_vs_per_call  the same step with one launch per conversion
served        Poisson arrivals of transfer-and-convert requests at fractions
              of the measured saturation rate: p50/p99 latency, throughput

--impl reference runs the CPU oracle as the reference arm on the same
workload and metric.  Under torchrun (N > 1) every rank runs an independent
replica (the path has no exchange step); value = all ranks' bytes / the
slowest rank's time.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_RECORDS = 200_000
BATCH = 16
BLOCK = 32
FALLBACK_HBM_GBS = 6400.0
METRIC = "layout-convert HBM GB/s"
KERNEL_SOURCES = ["paper_2511_04853_b300/csrc/mrn_kernels.cu", "paper_2511_04853_b300/csrc/mrn_device.cuh",
                  "paper_2511_04853_b300/csrc/mrn_plan.h"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--batch", type=int, default=BATCH)
    ap.add_argument("--device-only", action="store_true",
                    help="profiling runs: only the timed device step (no e2e, baselines or extras)")
    ap.add_argument("--case", default=None,
                    help="profiling runs: repeat one conversion, e.g. cells:aos:soa:16777216 "
                         "(schema:src[/B]:dst[/B]:records), or one overlapping move, memmove:bytes:shift")
    ap.add_argument("--mixed-jobs", type=int, default=4096,
                    help="collections in the mixed batch (0 skips it)")
    ap.add_argument("--mixed-only", action="store_true", help="run the mixed batch alone")
    ap.add_argument("--serve-rates", default="0.25,0.5,0.9,1.2",
                    help="served arrival rates as fractions of the measured saturation rate")
    return ap.parse_args()


def kernel_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def bytes_per_collection(stride=24, n=N_RECORDS):
    # three conversions, each reads and writes the collection once
    return 3 * 2 * n * stride


def workload_config(batch):
    return {"workload": "calorimeter cells: %d collections x 200,000 records (24-byte AoS: f32 energy, "
                        "time, eta, phi; u32 cell_id; u16 gain, quality); per collection AoS->SoA, "
                        "SoA->AoSoA(32), AoSoA(32)->AoS" % batch,
            "records_per_collection": N_RECORDS, "collections_per_step": batch,
            "launch": "one persistent kernel per step (CUDA graph replay)",
            "l2": "inputs larger than L2 (%d MB touched per step, L2 126 MB)"
                  % (batch * bytes_per_collection() // 10**6),
            "parallelism": "replicas"}


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc, self.lines = index, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                pw.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(pw) if pw else None}


# --------------------------------------------------------------- reference

def oracle_step_setup(n_records, seed=1):
    import datagen
    import oracle
    o = oracle.Schema(datagen.CELLS)
    d = datagen.workload("cells", n_records, seed)
    aos = oracle.pack(o, d, "aos")
    soa = oracle.convert(o, aos, "soa")
    blk = oracle.convert(o, soa, "aosoa", BLOCK)
    outs = [oracle.alloc(o, "soa", n_records), oracle.alloc(o, "aosoa", n_records, 0, BLOCK),
            oracle.alloc(o, "aos", n_records)]

    def step():
        for src, dst in zip([aos, soa, blk], outs):
            st, _ = oracle.convert_into(o, src, dst)
            assert st == 0
    return step


def cpu_oracle_rate(seconds, n_records):
    """The oracle (plain C, one thread) on the step's three conversions of
    one collection of n_records, repeated for about `seconds`; GB/s."""
    step = oracle_step_setup(n_records)
    reps, t0 = 0, time.perf_counter()
    while True:
        step()
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return reps * bytes_per_collection(24, n_records) / el / 1e9, reps, el


def _oracle_worker(job):
    """One host process of the all-cores oracle measurement: its own seeded
    collection, the three conversions repeated for `seconds` from a common
    start time."""
    seconds, n_records, seed, start_at = job
    step = oracle_step_setup(n_records, seed)
    step()
    while time.time() < start_at:
        time.sleep(0.01)
    reps, t0 = 0, time.perf_counter()
    while True:
        step()
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            return reps, el


def cpu_oracle_rate_all_cores(seconds, n_records):
    """The same oracle, unchanged, in one process per host core (spawned:
    the parent already holds a CUDA context), each on its own collection,
    all started together; aggregate GB/s."""
    import multiprocessing as mp
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    lead = 5.0 + 0.05 * cores
    start_at = time.time() + lead
    pool = ctx.Pool(cores)
    try:
        job = pool.map_async(_oracle_worker, [(seconds, n_records, 1 + i, start_at) for i in range(cores)])
        res = job.get(timeout=lead + seconds + 120.0)  # a worker that died must not hang the bench
    except Exception as e:
        pool.terminate()
        return None, "not measured: %s" % type(e).__name__
    pool.close()
    pool.join()
    per = bytes_per_collection(24, n_records)
    return sum(r * per / el for r, el in res) / 1e9, cores


def run_reference(args, rank, world):
    if rank != 0:
        return
    # size each step so the whole --steps/--warmup run stays near a minute
    probe, _, _ = cpu_oracle_rate(0.5, 20000)
    per_step_s = 60.0 / max(1, args.steps + args.warmup)
    n_rec = int(max(1000, min(N_RECORDS, per_step_s * probe * 1e9 / bytes_per_collection(24, 1))))
    step = oracle_step_setup(n_rec)
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t0
    val = args.steps * bytes_per_collection(24, n_rec) / el / 1e9
    sample = "%d-record cells collection x 3 conversions per step" % n_rec
    line = {"impl": "reference", "metric": METRIC, "value": round(val, 3), "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(el / args.steps * 1e3, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": workload_config(args.batch),
            "cpu_baseline": {"value": round(val, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(val, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------- mixed 4,096-job batch

MIXED_TARGETS = [("soa", 0), ("aosoa", 32), ("aosoa", 128)]
MIXED_SCHEMAS = ["points", "cells", "tracks"]


def mixed_plan(jobs, seed=3, lo=3.0, hi=6.0):
    """Job list of the mixed batch: sizes round(10^U(lo, hi)) records,
    schema uniform over points / cells / tracks, AoS source, target uniform
    over SoA / AoSoA(32) / AoSoA(128) (track parents in AoSoA(B) keep their
    offsets and child columns after the blocks)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    ns = np.rint(10.0 ** rng.uniform(lo, hi, jobs)).astype(np.int64)
    sch = rng.integers(0, 3, jobs)
    tgt = rng.integers(0, 3, jobs)
    return [(MIXED_SCHEMAS[sch[i]], int(ns[i]), MIXED_TARGETS[tgt[i]]) for i in range(jobs)]


def device_aos(torch, s, name, n, seed):
    """AoS source of one collection, generated on the device with the
    workload's value distributions (padding bytes zero).  Returns the record
    buffer, the child pool (tracks) and the child count."""
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    kw = {"device": "cuda", "generator": g}
    rec = torch.zeros(max(1, n * s.stride), dtype=torch.uint8, device="cuda")
    rv = rec[: n * s.stride].view(n, s.stride)
    off = {c["name"]: c["aos_offset"] for c in s.columns}

    def put(field, t):
        b = t.contiguous().view(torch.uint8).view(n, -1)
        rv[:, off[field]: off[field] + b.shape[1]].copy_(b)

    def uni(a, b):
        return torch.rand(n, **kw) * (b - a) + a

    def bits32(shape):
        return torch.randint(-2 ** 31, 2 ** 31, shape, dtype=torch.int64, **kw).to(torch.int32)

    def low16(t):
        return t.to(torch.int32).view(torch.uint8).view(n, 4)[:, :2]

    pool, m = None, 0
    if name == "points":
        put("x", uni(-1, 1)), put("y", uni(-1, 1)), put("z", uni(-1, 1))
        put("id", bits32((n,))), put("key", bits32((n, 2)))
        put("flag", torch.randint(0, 256, (n,), dtype=torch.uint8, **kw))
    elif name == "cells":
        put("energy", torch.empty(n, device="cuda").exponential_(2.0, generator=g))
        put("time", torch.randn(n, **kw) * 5.0)
        put("eta", uni(-4.9, 4.9)), put("phi", uni(-3.141592653589793, 3.141592653589793))
        put("cell_id", torch.randperm(n, **kw).to(torch.int32))
        put("gain", low16(torch.randint(0, 4, (n,), **kw)))
        put("quality", low16(torch.randint(0, 65536, (n,), **kw)))
    else:
        put("pt", torch.empty(n, device="cuda").exponential_(0.1, generator=g))
        put("eta", uni(-2.5, 2.5))
        put("label", torch.randint(0, 10, (n,), dtype=torch.int32, **kw))
        lens = torch.poisson(torch.full((n,), 20.0, device="cuda"), generator=g).clamp_(max=256).to(torch.int64)
        begs = torch.cumsum(lens, 0) - lens
        rv[:, s.info.jag_length_offset: s.info.jag_length_offset + 4].copy_(
            lens.to(torch.int32).view(torch.uint8).view(n, 4))
        rv[:, s.info.jag_begin_offset: s.info.jag_begin_offset + 8].copy_(begs.view(torch.uint8).view(n, 8))
        m = int(lens.sum().item())
        pool = torch.empty(max(1, m), 2, dtype=torch.int32, device="cuda")
        pool[:m, 0] = bits32((m,))
        pool[:m, 1] = torch.rand(m, **kw).view(torch.int32)
        pool = pool.view(torch.uint8).view(-1)
    return rec, pool, m


def run_mixed(mrn, torch, stream, peak, args):
    """The mixed batch (4,096 collections by default) in one persistent
    launch per step under a CUDA graph, with the autotuner's shapes and
    without them, against one launch per collection on the same stream."""
    import datagen
    plan = mixed_plan(args.mixed_jobs)
    schemas = {k: mrn.Schema(datagen.WORKLOAD_SCHEMAS[k]) for k in MIXED_SCHEMAS}
    pairs, outs, alg, alg_jag = [], [], 0, 0
    t_setup = time.perf_counter()
    for i, (name, n, (dk, db)) in enumerate(plan):
        s = schemas[name]
        rec, pool, m = device_aos(torch, s, name, n, 1000 + i)
        out = torch.empty(s.required_bytes(dk, n, m, db), dtype=torch.uint8, device="cuda")
        src = mrn.View(s, "aos", n, base=rec, child_pool=pool, m=m)
        dst = mrn.View(s, dk, n, block=db, base=out, m=m)
        pairs.append((src, dst))
        outs.append(out)
        if name == "tracks":
            alg += 24 * n + 8 * m + 12 * n + 4 * (n + 1) + 8 * m
            alg_jag += 24 * n + 8 * m + 12 * n + 4 * (n + 1) + 8 * m
        else:
            alg += n * (s.stride + sum(c["size"] for c in s.columns))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup

    def timed(fn, reps):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        assert mrn.sync() == mrn.OK
        return a.elapsed_time(b) / reps

    res = {"workload": "%d collections, records round(10^U(3,6)), schema uniform over points / cells / "
                       "tracks (jagged, Poisson(20) children clipped at 256), AoS source, target uniform over "
                       "SoA / AoSoA(32) / AoSoA(128)" % len(plan),
           "records": sum(n for _, n, _ in plan), "algorithmic_bytes": alg,
           "algorithmic_bytes_jagged_jobs": alg_jag, "setup_s": round(setup_s, 1)}
    # autotuner off: the library's default shapes
    mrn.autotune_clear()
    plain = mrn.Batch(pairs, use_graph=True)
    plain.launch()
    torch.cuda.synchronize()
    assert mrn.sync() == mrn.OK
    want = [o.clone() for o in outs]
    for o in outs:
        o.fill_(0xA5)
    ms_plain = timed(plain.launch, 5)
    del plain
    # one launch per collection, same kernels, same stream
    per = mrn.Batch(pairs, use_graph=False)
    for o in outs:
        o.fill_(0xA5)
    ms_per = timed(per.launch_per_job, 3)
    for o, w in zip(outs, want):
        assert torch.equal(o, w), "per-call output differs from the batched output"
    del per
    # autotuned shapes for every non-jagged (schema, target) pair
    tuned = {}
    for name in ("points", "cells"):
        for dk, db in MIXED_TARGETS:
            r = mrn.autotune(schemas[name], "aos", dk, 1 << 22, 0, db)
            tuned["%s_aos_to_%s%s" % (name, dk, db or "")] = {k: r[k] for k in ("staged", "threads",
                                                                               "tile_records", "ctas_per_sm")}
    tb = mrn.Batch(pairs, use_graph=True)
    launch_shape = tb.tune()
    for o in outs:
        o.fill_(0xA5)
    ms_tuned = timed(tb.launch, 5)
    for o, w in zip(outs, want):
        assert torch.equal(o, w), "autotuned batch output differs"
    del tb
    mrn.autotune_clear()
    best = min(ms_plain, ms_tuned)
    res.update({"ms_per_launch_default_shapes": round(ms_plain, 3),
                "ms_per_launch_autotuned": round(ms_tuned, 3),
                "gbps": round(alg / (best * 1e-3) / 1e9, 1),
                "frac_of_hbm": round(alg / (best * 1e-3) / 1e9 / peak, 3),
                "gbps_default_shapes": round(alg / (ms_plain * 1e-3) / 1e9, 1),
                "gbps_autotuned": round(alg / (ms_tuned * 1e-3) / 1e9, 1),
                "per_call_ms": round(ms_per, 3), "per_call_launches": len(plan),
                "speedup_vs_per_call": round(ms_per / best, 3),
                "autotuned_shapes": tuned, "autotuned_launch": launch_shape})
    del want, outs, pairs
    torch.cuda.empty_cache()
    return res


# -------------------------------------------------------------------- mine

def make_inputs(mrn, torch, s, batch):
    """R collections resident on the device: AoS, SoA and AoSoA(32) inputs
    and garbage-filled outputs.  Values come from the seeded generator; the
    layouts are built with the library's own kernels."""
    import datagen
    import numpy as np
    colls = []
    for i in range(batch):
        d = datagen.workload("cells", N_RECORDS, 1 + i)
        soa = torch.zeros(s.required_bytes("soa", N_RECORDS), dtype=torch.uint8, device="cuda")
        for c, v in enumerate(d["columns"]):
            off = s.soa_region_offset(N_RECORDS, 0, c)
            b = torch.from_numpy(np.ascontiguousarray(v).view(np.uint8)).cuda()
            soa[off: off + b.numel()].copy_(b)
        aos = torch.empty(s.required_bytes("aos", N_RECORDS), dtype=torch.uint8, device="cuda")
        blk = torch.empty(s.required_bytes("aosoa", N_RECORDS, 0, BLOCK), dtype=torch.uint8, device="cuda")
        mrn.convert(mrn.View(s, "soa", N_RECORDS, base=soa), mrn.View(s, "aos", N_RECORDS, base=aos))
        mrn.convert(mrn.View(s, "soa", N_RECORDS, base=soa),
                    mrn.View(s, "aosoa", N_RECORDS, block=BLOCK, base=blk))
        outs = [torch.full_like(soa, 0xA5), torch.full_like(blk, 0xA5), torch.full_like(aos, 0xA5)]
        colls.append({"aos": aos, "soa": soa, "blk": blk, "out": outs})
    assert mrn.sync() == mrn.OK
    return colls


def pairs_for(mrn, s, colls):
    n = N_RECORDS
    out = []
    for c in colls:
        out.append((mrn.View(s, "aos", n, base=c["aos"]), mrn.View(s, "soa", n, base=c["out"][0])))
        out.append((mrn.View(s, "soa", n, base=c["soa"]), mrn.View(s, "aosoa", n, block=BLOCK, base=c["out"][1])))
        out.append((mrn.View(s, "aosoa", n, block=BLOCK, base=c["blk"]), mrn.View(s, "aos", n, base=c["out"][2])))
    return out


def check_outputs(torch, colls):
    """Each output must equal the input that mirrors it (bit-exact): the
    three conversions of a collection form a cycle."""
    for c in colls:
        assert torch.equal(c["out"][0], c["soa"]), "AoS->SoA output differs from the SoA input"
        assert torch.equal(c["out"][1], c["blk"]), "SoA->AoSoA output differs from the AoSoA input"
        assert torch.equal(c["out"][2], c["aos"]), "AoSoA->AoS output differs from the AoS input"


def traffic_record():
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        j = json.load(f)
    if j.get("kernel_source_hash") != kernel_hash():
        return None
    return j


def run_mine(args, rank, world):
    import torch
    import torch.distributed as dist
    import paper_2511_04853_b300 as mrn
    import datagen

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    s = mrn.Schema(datagen.CELLS)
    colls = make_inputs(mrn, torch, s, args.batch)
    batch = mrn.Batch(pairs_for(mrn, s, colls), use_graph=True)
    launch_shape = batch.tune()  # the batch autotuner picks the launch shape (setup, not timed)
    step_bytes = args.batch * bytes_per_collection()

    def barrier():
        if world > 1:
            dist.barrier()

    # the measured path is checked before it is timed
    batch.launch()
    assert mrn.sync() == mrn.OK
    check_outputs(torch, colls)

    # ---- device step: one persistent launch (graph replay) per step
    for _ in range(args.warmup):
        batch.launch()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    # per-launch events bracket every 16th launch (the kernel's launch
    # duration for the roofline); the others run back to back
    sampled = list(range(0, args.steps, 16))
    ev = {k: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for k in sampled}
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        if k in ev:
            ev[k][0].record(stream)
            batch.launch()
            ev[k][1].record(stream)
        else:
            batch.launch()
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = clk.stop()
    total_ms = t_start.elapsed_time(t_end)
    launch_ms = [a.elapsed_time(b) for a, b in ev.values()]
    ms_step = total_ms / args.steps
    if world > 1:
        t = torch.tensor([ms_step], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    value = world * step_bytes / (ms_step * 1e-3) / 1e9
    assert mrn.sync() == mrn.OK
    check_outputs(torch, colls)

    if args.device_only:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 5),
                              "mode": "device-only (profiling)", "config": workload_config(args.batch)}),
                  flush=True)
        return

    extra = {}
    if rank == 0:
        # ---- per-call baseline: the same 3R conversions, one launch each
        for _ in range(3):
            batch.launch_per_job()
        torch.cuda.synchronize()
        reps = max(3, min(50, args.steps // 10))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            batch.launch_per_job()
        b.record(stream)
        torch.cuda.synchronize()
        per_call_ms = a.elapsed_time(b) / reps
        assert mrn.sync() == mrn.OK
        check_outputs(torch, colls)
        extra["batched_vs_per_call"] = {"per_call_ms_per_step": round(per_call_ms, 4),
                                        "batched_ms_per_step": round(ms_step, 4),
                                        "speedup": round(per_call_ms / ms_step, 3),
                                        "per_call_launches_per_step": 3 * args.batch}

    # ---- end to end through pinned host buffers
    e2e = run_e2e(mrn, torch, s, colls, args, world)
    del batch
    if rank != 0:
        return
    for c in colls:
        c["out"] = None
    peak, peak_src = peaks()
    lm = statistics.mean(launch_ms)
    achieved = step_bytes / (lm * 1e-3) / 1e9
    tr = traffic_record()
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": tr["bytes_per_launch"] if tr else None,
            "kernel": "k_batch (persistent; %d conversions per launch)" % (3 * args.batch),
            "algorithmic_bytes_per_launch": step_bytes, "launch_ms_mean": round(lm, 5),
            "launch_ms_median": round(statistics.median(launch_ms), 5),
            "launch_samples": "%d of %d timed launches bracketed by events" % (len(launch_ms), args.steps),
            "peak_source": ("of measured (MEASURED_PEAKS.json hbm_gbs, copy read+write)" if peak_src == "measured"
                            else "of fallback 6.4 TB/s")}
    del colls
    torch.cuda.empty_cache()
    extra.update(secondary(mrn, torch, stream, peak))
    if args.mixed_jobs > 0:
        extra["batched_mixed"] = run_mixed(mrn, torch, stream, peak, args)
    extra["sensor_grid"] = run_sensor_grid(mrn, torch, stream)
    extra["collection_ops"] = run_collection_ops(mrn, torch, stream, peak)
    extra["served"] = run_served(mrn, torch, args)
    cpu_val, cpu_reps, cpu_s = cpu_oracle_rate(10.0, N_RECORDS)
    cpu_all, cpu_cores = cpu_oracle_rate_all_cores(10.0, N_RECORDS)
    line = {"metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic (seeded generator; distributions of the calorimeter-cell workload)",
            "config": workload_config(args.batch),
            "batch_launch": dict(launch_shape, chosen_by="mrn_batch_tune (chunk x CTAs per SM, timed on the batch)"),
            "e2e": e2e,
            "gpu_launches": args.steps,
            "roofline": roof,
            "cpu_baseline": {"value": round(cpu_val, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": "3 conversions of one 200,000-record collection x %d (%.1f s)"
                                       % (cpu_reps, cpu_s),
                             "all_cores": {"value": round(cpu_all, 3) if cpu_all else None, "unit": "GB/s",
                                           "cores": cpu_cores,
                                           "sample": "one process per core, each the same 3 conversions of "
                                                     "its own 200,000-record collection for 10 s, started "
                                                     "together; aggregate"}},
            "clocks": clocks}
    line.update(extra)
    print(json.dumps(line), flush=True)


def run_e2e(mrn, torch, s, colls, args, world, n_streams=2, chunk_bytes=0):
    """Host pinned AoS -> device SoA, SoA -> AoSoA(32), device AoSoA(32) ->
    host pinned AoS for every collection of the batch, per step."""
    n = N_RECORDS
    h_in = [c["aos"].cpu().pin_memory() for c in colls]
    h_out = [torch.empty_like(h).pin_memory() for h in h_in]
    d_soa = [torch.empty_like(c["soa"]) for c in colls]
    d_blk = [torch.empty_like(c["blk"]) for c in colls]
    views = []
    for i in range(len(colls)):
        views.append((mrn.View(s, "aos", n, base=h_in[i], mem="pinned"), mrn.View(s, "soa", n, base=d_soa[i]),
                      mrn.View(s, "aosoa", n, block=BLOCK, base=d_blk[i]),
                      mrn.View(s, "aos", n, base=h_out[i], mem="pinned")))

    streams = [torch.cuda.Stream() for _ in range(n_streams)]
    main = torch.cuda.current_stream()

    def step():
        # collection i on stream i % n_streams: collections' device -> host
        # copies overlap later ones' host -> device copies (each direction
        # has its own copy pipeline; a stream only orders its own
        # collections)
        for st in streams:
            st.wait_stream(main)
        for i, (hin, soa, blk, hout) in enumerate(views):
            st = streams[i % len(streams)]
            mrn.transfer_convert(hin, soa, chunk_bytes=chunk_bytes, stream=st)
            mrn.convert(soa, blk, stream=st)
            mrn.transfer_convert(blk, hout, chunk_bytes=chunk_bytes, stream=st)
        for st in streams:
            main.wait_stream(st)

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    for i in range(len(colls)):
        assert torch.equal(h_out[i], h_in[i]), "end-to-end round trip differs"
    k = max(3, min(20, args.steps // 100))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(k):
        step()
    torch.cuda.synchronize()
    el = (time.perf_counter() - t0) / k
    assert mrn.sync() == mrn.OK
    step_bytes = len(colls) * bytes_per_collection()
    return {"value": round(world * step_bytes / el / 1e9, 2), "unit": "GB/s",
            "h2d_bytes_per_step": len(colls) * n * 24, "d2h_bytes_per_step": len(colls) * n * 24,
            "ms_per_step": round(el * 1e3, 3), "steps": k,
            "path": "mrn_transfer_convert (default 4 MiB chunks, 4 slots) + mrn_convert, pinned host buffers, "
                    "collection i on stream i %% %d" % n_streams}


def secondary(mrn, torch, stream, peak):
    """Single-collection launches at the workload sizes and scale-up
    collections (2^26 records), L2 flushed before each launch, against the
    HBM roofline; the host link bandwidth."""
    import numpy as np
    import datagen
    out = {}
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def time_conv(src, dst, reps):
        ts = []
        for i in range(reps + 2):
            flush.fill_(i & 0xff)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            mrn.convert(src, dst)
            b.record(stream)
            b.synchronize()
            if i >= 2:
                ts.append(a.elapsed_time(b))
        return statistics.median(ts), sorted(ts)[:max(1, len(ts) // 5)]

    def row(alg, med, fastest):
        return {"us_median": round(med * 1e3, 2), "gbps": round(alg / (med * 1e-3) / 1e9, 1),
                "frac_of_hbm": round(alg / (med * 1e-3) / 1e9 / peak, 3),
                "gbps_mean_fastest_fifth": round(alg / (statistics.mean(fastest) * 1e-3) / 1e9, 1)}

    rows = {}
    for name, n, pairs in [("points", 10000, [("aos", 0, "soa", 0), ("soa", 0, "aos", 0)]),
                           ("cells", 200000, [("aos", 0, "soa", 0), ("soa", 0, "aosoa", 32),
                                              ("aosoa", 32, "aos", 0)]),
                           ("cells", 1 << 26, [("aos", 0, "soa", 0), ("soa", 0, "aos", 0),
                                               ("soa", 0, "aosoa", 32), ("aosoa", 32, "aos", 0)]),
                           ("points", 1 << 26, [("aos", 0, "soa", 0), ("soa", 0, "aos", 0)])]:
        s = mrn.Schema(datagen.WORKLOAD_SCHEMAS[name])
        bufs = {}
        for sk, sb, dk, db in pairs:
            for k, bk in ((sk, sb), (dk, db)):
                if (k, bk) not in bufs:
                    bufs[(k, bk)] = torch.full((s.required_bytes(k, n, 0, bk),), 0x3C, dtype=torch.uint8,
                                               device="cuda")
        for sk, sb, dk, db in pairs:
            src = mrn.View(s, sk, n, block=sb, base=bufs[(sk, sb)])
            dst = mrn.View(s, dk, n, block=db, base=bufs[(dk, db)])
            med, fastest = time_conv(src, dst, 10 if n > 1e6 else 30)
            key = "%s_%d_%s%s_to_%s%s" % (name, n, sk, sb or "", dk, db or "")
            rows[key] = row(2 * n * s.stride, med, fastest)
        del bufs
    # jagged tracks, AoS -> SoA and back (canonical child pool)
    s = mrn.Schema(datagen.TRACKS)
    for n in (100000, 1 << 22):
        m, recs, pool = jagged_aos(torch, s, n)
        soa = torch.empty(s.required_bytes("soa", n, m), dtype=torch.uint8, device="cuda")
        src = mrn.View(s, "aos", n, base=recs, child_pool=pool, m=m)
        dst = mrn.View(s, "soa", n, base=soa, m=m)
        alg = n * 24 + m * 8 + n * 12 + (n + 1) * 4 + m * 8
        med, fastest = time_conv(src, dst, 10)
        rows["tracks_%d_aos_to_soa" % n] = dict(row(alg, med, fastest), children=m)
        back = mrn.View(s, "aos", n, base=recs, child_pool=pool, m=m)
        med, fastest = time_conv(dst, back, 10)
        rows["tracks_%d_soa_to_aos" % n] = row(alg, med, fastest)
        assert mrn.sync() == mrn.OK
        del recs, pool, soa
    out["single_collection"] = rows
    del flush
    # transfer-and-convert: chunked staging against zero-copy (the kernel
    # reads / writes the pinned host buffer itself), source bytes per second
    s = mrn.Schema(datagen.CELLS)
    abl = {}
    for n in (200000, 1 << 24):
        h_aos = torch.full((n * 24,), 0x3C, dtype=torch.uint8).pin_memory()
        d_soa = torch.empty(s.required_bytes("soa", n), dtype=torch.uint8, device="cuda")
        hv = mrn.View(s, "aos", n, base=h_aos, mem="pinned")
        dv = mrn.View(s, "soa", n, base=d_soa)
        for name, zc in (("chunked", False), ("zero_copy", True)):
            for direction, a, b in (("h2d", hv, dv), ("d2h", dv, hv)):
                reps = 20 if n < 1e6 else 5
                mrn.transfer_convert(a, b, stream=stream, zero_copy=zc)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for _ in range(reps):
                    mrn.transfer_convert(a, b, stream=stream, zero_copy=zc)
                torch.cuda.synchronize()
                el = (time.perf_counter() - t0) / reps
                abl["cells_%d_%s_%s_gbps" % (n, direction, name)] = round(n * 24 / el / 1e9, 1)
        assert mrn.sync() == mrn.OK
        del h_aos, d_soa
    out["transfer_chunked_vs_zero_copy"] = abl
    # host link: pinned 1 GiB copies, best of 5
    h = torch.empty(1 << 30, dtype=torch.uint8).pin_memory()
    dbuf = torch.empty(1 << 30, dtype=torch.uint8, device="cuda")
    best_h2d = best_d2h = 1e9
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        dbuf.copy_(h, non_blocking=True)
        b.record(stream)
        b.synchronize()
        best_h2d = min(best_h2d, a.elapsed_time(b))
        a.record(stream)
        h.copy_(dbuf, non_blocking=True)
        b.record(stream)
        b.synchronize()
        best_d2h = min(best_d2h, a.elapsed_time(b))
    # both directions at once (two streams): the ceiling of a round trip
    h2 = torch.empty(1 << 30, dtype=torch.uint8).pin_memory()
    dbuf2 = torch.empty(1 << 30, dtype=torch.uint8, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    best_bi = 1e9
    for _ in range(5):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(s1):
            dbuf.copy_(h, non_blocking=True)
        with torch.cuda.stream(s2):
            h2.copy_(dbuf2, non_blocking=True)
        torch.cuda.synchronize()
        best_bi = min(best_bi, time.perf_counter() - t0)
    out["host_link_gbps"] = {"h2d": round((1 << 30) / (best_h2d * 1e-3) / 1e9, 1),
                             "d2h": round((1 << 30) / (best_d2h * 1e-3) / 1e9, 1),
                             "both_directions_total": round(2 * (1 << 30) / best_bi / 1e9, 1)}
    del h2, dbuf2
    del h, dbuf
    torch.cuda.empty_cache()
    return out


def run_collection_ops(mrn, torch, stream, peak):
    """Size-changing operations on device collections (the overlapping move
    k_move underneath), against the HBM roofline: algorithmic bytes are the
    bytes moved read once and written once (plus a conversion's own bytes
    for an insert), timed with CUDA events around each call."""
    import datagen
    out = {}

    def timed(fn, reps=5):
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        assert mrn.sync() == mrn.OK
        return statistics.median(ts)

    def row(alg, ms):
        return {"ms": round(ms, 4), "gbps": round(alg / (ms * 1e-3) / 1e9, 1),
                "frac_of_hbm": round(alg / (ms * 1e-3) / 1e9 / peak, 3)}

    # the overlapping move alone: 1 GiB shifted by a little and by a lot
    nb = 1 << 30
    buf = torch.empty(nb + (64 << 20), dtype=torch.uint8, device="cuda")
    p0 = buf.data_ptr() + (32 << 20)
    mv = {}
    for name, shift in (("up_64B", 64), ("down_64B", -64), ("up_8MiB", 8 << 20), ("down_8MiB", -(8 << 20))):
        ms = timed(lambda: mrn.memmove(p0 + shift, p0, nb, stream=stream))
        mv[name] = row(2 * nb, ms)
    out["memmove_1GiB"] = mv
    del buf
    # a calorimeter-cell SoA collection of 2^26 objects: erase 1% at the
    # front, insert 1% (from device AoS) at the front
    s = mrn.Schema(datagen.CELLS)
    n, k = 1 << 26, (1 << 26) // 100
    coll = mrn.Collection(s, "soa", capacity=n + k)
    coll.resize(n)
    src = torch.full((k * 24,), 0x3C, dtype=torch.uint8, device="cuda")
    sv = mrn.View(s, "aos", k, base=src)
    cells = {}
    ms_e, ms_i = [], []
    for _ in range(4):
        ms_e.append(timed(lambda: coll.erase(0, k), 1))
        ms_i.append(timed(lambda: coll.insert(0, sv), 1))
    cells["erase_front_1pct"] = row(2 * (n - k) * 24, statistics.median(ms_e))
    cells["insert_front_1pct"] = row(2 * (n - k) * 24 + 2 * k * 24, statistics.median(ms_i))
    out["cells_soa_2^26"] = cells
    del coll, src
    # jagged tracks, SoA collection of 4,194,304 parents (~84 M children)
    s = mrn.Schema(datagen.TRACKS)
    n = 1 << 22
    m, recs, pool = jagged_aos(torch, s, n)
    coll = mrn.Collection(s, "soa", capacity=n + n // 50, child_capacity=m + m // 20)
    coll.assign(mrn.View(s, "aos", n, base=recs, child_pool=pool, m=m))
    k = n // 100
    kv = mrn.View(s, "aos", k, base=recs, child_pool=pool, m=m)
    tr = {}
    ms_e, ms_i, moved = [], [], []
    for _ in range(3):
        n0, m0 = coll.sizes()[:2]
        ms_e.append(timed(lambda: coll.erase(0, k), 1))
        n1, m1 = coll.sizes()[:2]
        moved.append((n1 * 12 + (n1 + 1) * 4 + m1 * 8, m0 - m1))
        ms_i.append(timed(lambda: coll.insert(0, kv), 1))
    b_move, kids = moved[0]
    tr["erase_front_1pct"] = dict(row(2 * b_move, statistics.median(ms_e)), children_removed=int(kids))
    tr["insert_front_1pct"] = dict(row(2 * b_move + k * 24 + kids * 8 + k * 16 + kids * 8,
                                       statistics.median(ms_i)))
    tr["note"] = ("field-major jagged erase / insert wait for the stream to read offsets (and an AoS "
                  "source's child count); those host round trips are inside the timed call")
    out["tracks_soa_4M"] = tr
    del coll, recs, pool
    torch.cuda.empty_cache()
    return out


def run_sensor_grid(mrn, torch, stream):
    """The paper's sensor workload (Sec. VII, Listing 1 Sensor records) as a
    synthetic grid: host AoS sensors -> device SoA (transfer-and-convert), a
    stand-in per-sensor computation on the SoA columns (energy = counts * A
    + B, zero for noisy sensors; the real calibration is not in the paper),
    device SoA -> host AoS.  Reports each stage against a single-threaded
    numpy pass over the same AoS array."""
    import numpy as np
    import datagen
    s = mrn.Schema(datagen.SENSOR)
    off = {c["name"]: c["aos_offset"] for c in s.columns}
    col = {c["name"]: i for i, c in enumerate(s.columns)}
    rows = {}
    for g in (100, 1000, 3000, 5000):
        n = g * g
        rng = np.random.default_rng(g)
        rec = np.zeros((n, s.stride), np.uint8)
        rec[:, off["type"]] = rng.integers(0, 4, n, dtype=np.uint8)
        rec[:, off["counts"]: off["counts"] + 8] = rng.integers(0, 1 << 16, n, dtype=np.uint64).view(np.uint8).reshape(n, 8)
        rec[:, off["calibration_data.noisy"]] = (rng.random(n) < 0.01).astype(np.uint8)
        for k, lo, hi in (("parameter_A", 0.9, 1.1), ("parameter_B", -1.0, 1.0), ("noise_A", 0.0, 0.1),
                          ("noise_B", 0.0, 0.1)):
            o = off["calibration_data." + k]
            rec[:, o: o + 4] = rng.uniform(lo, hi, n).astype(np.float32).view(np.uint8).reshape(n, 4)
        h_in = torch.from_numpy(rec.reshape(-1)).pin_memory()
        h_out = torch.empty_like(h_in).pin_memory()
        soa = torch.empty(s.required_bytes("soa", n), dtype=torch.uint8, device="cuda")

        def column(name, dtype):
            o = s.soa_region_offset(n, 0, col[name])
            size = torch.tensor([], dtype=dtype).element_size()
            return soa[o: o + n * size].view(dtype)

        hv = mrn.View(s, "aos", n, base=h_in, mem="pinned")
        dv = mrn.View(s, "soa", n, base=soa)
        hv_out = mrn.View(s, "aos", n, base=h_out, mem="pinned")
        counts, energy = column("counts", torch.int64), column("energy", torch.float32)
        a, b = column("calibration_data.parameter_A", torch.float32), column("calibration_data.parameter_B", torch.float32)
        noisy = column("calibration_data.noisy", torch.uint8)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        best = None
        for _ in range(3):
            ev[0].record(stream)
            mrn.transfer_convert(hv, dv, stream=stream)
            ev[1].record(stream)
            energy.copy_(torch.where(noisy != 0, 0.0, counts.to(torch.float32) * a + b))
            ev[2].record(stream)
            mrn.transfer_convert(dv, hv_out, stream=stream)
            ev[3].record(stream)
            torch.cuda.synchronize()
            t = [ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3])]
            if best is None or sum(t) < sum(best):
                best = t
        assert mrn.sync() == mrn.OK
        # the same computation on the host AoS array, one numpy pass
        t0 = time.perf_counter()
        cnt = rec[:, off["counts"]: off["counts"] + 8].copy().view(np.int64).reshape(-1)
        pa = rec[:, off["calibration_data.parameter_A"]:][:, :4].copy().view(np.float32).reshape(-1)
        pb = rec[:, off["calibration_data.parameter_B"]:][:, :4].copy().view(np.float32).reshape(-1)
        nz = rec[:, off["calibration_data.noisy"]]
        e_cpu = np.where(nz != 0, np.float32(0), cnt.astype(np.float32) * pa + pb).astype(np.float32)
        cpu_ms = (time.perf_counter() - t0) * 1e3
        out = h_out.numpy().reshape(n, s.stride)
        e_gpu = out[:, off["energy"]: off["energy"] + 4].copy().view(np.float32).reshape(-1)
        assert np.allclose(e_gpu, e_cpu, rtol=1e-6, atol=1e-6), "sensor energies differ"
        assert np.array_equal(np.delete(out, np.s_[off["energy"]: off["energy"] + 4], axis=1),
                              np.delete(rec, np.s_[off["energy"]: off["energy"] + 4], axis=1))
        rows["%dx%d" % (g, g)] = {"sensors": n, "h2d_convert_ms": round(best[0], 3),
                                  "stand_in_kernel_ms": round(best[1], 3), "d2h_convert_ms": round(best[2], 3),
                                  "gpu_total_ms": round(sum(best), 3), "cpu_numpy_ms": round(cpu_ms, 3),
                                  "transfer_convert_share": round((best[0] + best[2]) / sum(best), 3)}
        del h_in, h_out, soa
    torch.cuda.empty_cache()
    return {"what": "Sensor records (40-byte AoS) host -> device SoA -> stand-in energy pass -> host AoS, "
                    "against one numpy pass on the host AoS array", "grids": rows}


def run_served(mrn, torch, args):
    """Poisson arrivals of transfer-and-convert requests: source sizes
    log-uniform 10 KB - 256 MB, schemas points / cells / tracks, random
    source and target layouts, host->device or device->host, 64 GB budget.
    The saturation rate is measured first (a closed burst), then each
    fraction of it is offered for up to 3 s / 1500 requests."""
    import numpy as np
    import datagen
    rng = np.random.default_rng(4)
    kinds = [("aos", 0), ("soa", 0), ("aosoa", 32), ("aosoa", 128)]
    max_bytes = 256 << 20
    pools = {}
    for name in ("points", "cells"):
        s = mrn.Schema(datagen.WORKLOAD_SCHEMAS[name])
        nmax = max_bytes // s.stride
        hb, db = {}, {}
        for k, b in kinds:
            nb = s.required_bytes(k, nmax, 0, b)
            hb[(k, b)] = torch.full((nb,), 1, dtype=torch.uint8).pin_memory()
            db[(k, b)] = torch.full((nb,), 2, dtype=torch.uint8, device="cuda")
        pools[name] = (s, nmax, hb, db)
    # tracks: canonical AoS parents + pool on host, per-column SoA on device
    st = mrn.Schema(datagen.TRACKS)
    nt = 4_000_000
    dt = datagen.workload("tracks", nt, 9)
    lens = dt["lengths"].astype(np.uint64)
    csum = np.concatenate([[0], np.cumsum(lens)])
    recs = np.zeros((nt, 24), np.uint8)
    recs[:, 12:16] = lens.astype(np.uint32).view(np.uint8).reshape(nt, 4)
    recs[:, 16:24] = csum[:-1].astype(np.uint64).view(np.uint8).reshape(nt, 8)
    mt = int(csum[-1])
    t_host = (torch.from_numpy(recs.reshape(-1)).pin_memory(), torch.zeros(mt * 8, dtype=torch.uint8).pin_memory())
    t_cols = [torch.zeros(nt * 4, dtype=torch.uint8, device="cuda") for _ in range(3)]
    t_offs = torch.from_numpy(csum.astype(np.uint32).view(np.uint8)).cuda()
    t_kids = [torch.zeros(mt * 4, dtype=torch.uint8, device="cuda") for _ in range(2)]
    t_dev_dst = {k: torch.empty(st.required_bytes(k[0], nt, mt, k[1]), dtype=torch.uint8, device="cuda")
                 for k in (("soa", 0), ("aosoa", 32), ("aosoa", 128))}

    def make_request():
        name = ["points", "cells", "tracks"][rng.integers(0, 3)]
        size = int(10 ** rng.uniform(np.log10(10e3), np.log10(max_bytes)))
        h2d = rng.integers(0, 2) == 0
        if name == "tracks":
            n = max(1, min(nt - 1, size // 184))  # ~184 source bytes per parent at mean length 20
            m = int(csum[n])
            if h2d:
                dk, dbk = [("soa", 0), ("aosoa", 32), ("aosoa", 128)][rng.integers(0, 3)]
                src = mrn.View(st, "aos", n, base=t_host[0], child_pool=t_host[1], m=m, mem="pinned")
                dst = mrn.View(st, dk, n, block=dbk, base=t_dev_dst[(dk, dbk)], m=m)
            else:
                src = mrn.View(st, "soa", n, columns=t_cols, offsets=t_offs, child_columns=t_kids, m=m)
                dst = mrn.View(st, "aos", n, base=t_host[0], child_pool=t_host[1], m=m, mem="pinned")
            return src, dst, n * 24 + m * 8
        s, nmax, hb, db = pools[name]
        n = max(1, min(nmax, size // s.stride))
        sk, sb = kinds[rng.integers(0, 4)]
        dk, dbk = kinds[rng.integers(0, 4)]
        if h2d:
            src = mrn.View(s, sk, n, block=sb, base=hb[(sk, sb)], mem="pinned")
            dst = mrn.View(s, dk, n, block=dbk, base=db[(dk, dbk)])
        else:
            src = mrn.View(s, sk, n, block=sb, base=db[(sk, sb)])
            dst = mrn.View(s, dk, n, block=dbk, base=hb[(dk, dbk)], mem="pinned")
        return src, dst, n * s.stride

    budget = 64 << 30
    out = {"budget_bytes": budget, "slots": 8, "chunk_bytes": 4 << 20,
           "sizes": "log-uniform 10 KB - 256 MB of source", "schemas": "points, cells, tracks",
           "directions": "host->device, device->host"}
    # saturation: a closed burst of 400 requests
    sv = mrn.Server(budget, max_slots=8, chunk_bytes=4 << 20)
    reqs = [make_request() for _ in range(400)]
    t0 = time.perf_counter()
    tickets = [sv.submit(a, b)[1] for a, b, _ in reqs]
    for t in tickets:
        assert sv.wait(t, 600.0) == mrn.OK
    el = time.perf_counter() - t0
    sat = len(reqs) / el
    total = sum(x for _, _, x in reqs)
    out["saturation"] = {"req_per_s": round(sat, 1), "source_gbps": round(total / el / 1e9, 2)}
    sv.close()
    rates = []
    for frac in [float(x) for x in args.serve_rates.split(",") if x]:
        lam = frac * sat
        sv = mrn.Server(budget, max_slots=8, chunk_bytes=4 << 20)
        nreq = int(min(1500, max(50, lam * 3.0)))
        arrivals = np.cumsum(rng.exponential(1.0 / lam, nreq))
        batch = [make_request() for _ in range(nreq)]
        tickets, late = [], 0.0
        t0 = time.perf_counter()
        for (src, dst, _), ta in zip(batch, arrivals):
            now = time.perf_counter() - t0
            if ta > now:
                time.sleep(ta - now)
            else:
                late = max(late, now - ta)
            rc, t = sv.submit(src, dst)
            if rc == mrn.OK:
                tickets.append(t)
        for t in tickets:
            assert sv.wait(t, 600.0) == mrn.OK
        el = time.perf_counter() - t0
        stt = sv.stats()
        sv.close()
        rates.append({"frac_of_saturation": frac, "offered_req_per_s": round(lam, 1), "requests": nreq,
                      "p50_ms": round(stt["p50_ms"], 3), "p99_ms": round(stt["p99_ms"], 3),
                      "max_ms": round(stt["max_ms"], 3),
                      "throughput_source_gbps": round(stt["bytes_in"] / el / 1e9, 2),
                      "completed": stt["completed"], "rejected": stt["rejected"],
                      "peak_device_bytes": stt["peak_device_bytes"],
                      "client_max_lateness_ms": round(late * 1e3, 3)})
    out["rates"] = rates
    del pools, t_host, t_cols, t_offs, t_kids, t_dev_dst
    torch.cuda.empty_cache()
    return out


def run_case(args):
    """Repeats one conversion (for profilers): schema:src:dst:records, a
    layout written as aosoa/32 for blocks.  For the jagged tracks schema the
    AoS side is a canonical pool (Poisson(20) children clipped at 256)."""
    import torch
    import paper_2511_04853_b300 as mrn
    import datagen
    if args.case.startswith("memmove:"):
        # memmove:bytes:shift -- one overlapping move inside a device buffer
        _, nb, shift = args.case.split(":")
        nb, shift = int(nb), int(shift)
        buf = torch.empty(nb + 2 * abs(shift) + 256, dtype=torch.uint8, device="cuda")
        src = buf.data_ptr() + abs(shift) + 128
        for _ in range(args.warmup):
            mrn.memmove(src + shift, src, nb)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            mrn.memmove(src + shift, src, nb)
        e1.record()
        torch.cuda.synchronize()
        assert mrn.sync() == mrn.OK
        ms = e0.elapsed_time(e1) / args.steps
        print(json.dumps({"case": args.case, "ms": round(ms, 5), "gbps": round(2 * nb / (ms * 1e-3) / 1e9, 1)}),
              flush=True)
        return
    name, sk, dk, n = args.case.split(":")
    n = int(n)

    def lay(x):
        k, _, b = x.partition("/")
        return k, int(b or 0)
    (sk, sb), (dk, db) = lay(sk), lay(dk)
    s = mrn.Schema(datagen.WORKLOAD_SCHEMAS[name])
    if s.has_jagged:
        m, aos, pool = jagged_aos(torch, s, n)
        soa = torch.empty(s.required_bytes("soa", n, m), dtype=torch.uint8, device="cuda")
        a_view = mrn.View(s, "aos", n, base=aos, child_pool=pool, m=m)
        s_view = mrn.View(s, "soa", n, base=soa, m=m)
        src, dst = (a_view, s_view) if sk == "aos" else (s_view, a_view)
        if sk != "aos":
            mrn.convert(a_view, s_view)
        nbytes = n * 24 + m * 8 + n * 12 + (n + 1) * 4 + m * 8
    else:
        a = torch.full((s.required_bytes(sk, n, 0, sb),), 0x3C, dtype=torch.uint8, device="cuda")
        b = torch.empty(s.required_bytes(dk, n, 0, db), dtype=torch.uint8, device="cuda")
        src, dst = mrn.View(s, sk, n, block=sb, base=a), mrn.View(s, dk, n, block=db, base=b)
        nbytes = 2 * n * s.stride
    for _ in range(args.warmup):
        mrn.convert(src, dst)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        mrn.convert(src, dst)
    e1.record()
    torch.cuda.synchronize()
    assert mrn.sync() == mrn.OK
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"case": args.case, "ms": round(ms, 5),
                      "gbps": round(nbytes / (ms * 1e-3) / 1e9, 1)}), flush=True)


def jagged_aos(torch, s, n, seed=2):
    """Jagged AoS parents (tracks record: length at 12, begin at 16) with a
    canonical child pool, lengths min(Poisson(20), 256) from the seeded
    generator; returns (children, records, pool)."""
    import numpy as np
    import datagen
    d = datagen.workload("tracks", n, seed)
    m = d["m"]
    recs = torch.zeros(max(1, n * 24), dtype=torch.uint8, device="cuda")
    lens = torch.from_numpy(d["lengths"].astype(np.int32)).cuda()
    begs = torch.cumsum(lens.to(torch.int64), 0) - lens.to(torch.int64)
    rv = recs[: n * 24].view(n, 24)
    rv[:, 12:16].copy_(lens.view(torch.uint8).view(n, 4))
    rv[:, 16:24].copy_(begs.view(torch.uint8).view(n, 8))
    pool = torch.full((max(1, m * 8),), 7, dtype=torch.uint8, device="cuda")
    return m, recs, pool


def main():
    args = parse()
    if args.case:
        run_case(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.mixed_only:
        import torch
        import paper_2511_04853_b300 as mrn
        print(json.dumps(run_mixed(mrn, torch, torch.cuda.current_stream(), peaks()[0], args)), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    run_mine(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
