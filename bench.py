"""Benchmark of the layout-conversion hot path on one B300 (or N replicas).

Step: one replay of the CUDA graph of the mixed batch -- 4,096 collections
(records round(10^U(3, 6)), seed 3; schema uniform over points / cells /
tracks, the tracks jagged with Poisson(20) children clipped at 256; AoS
source; target uniform over SoA / AoSoA(32) / AoSoA(128)) converted in
three launches: the persistent k_batch twice (first the tracks' parents,
their begins written as offsets and each child pool checked, record by
record, to be canonical, with a share of the points / cells jobs; then
every canonical tracks pool as a plain conversion of the child schema,
with the other points / cells jobs), and k_batch_jag_rest (converts whole
again any tracks job whose pool is not canonical; none here, so it returns
at once).  About 92 GB of algorithmic bytes per step, inputs resident in
HBM (far larger than the 126 MB L2).

value         algorithmic bytes (read + write of every conversion) / step
              time (CUDA events around all timed steps)
roofline      the dominant kernel (k_batch, which moves every algorithmic
              byte) against the measured HBM copy bandwidth, from events
              recorded inside every timed replay after the scratch
              reset; per_kernel gives both parts
e2e           the same collections through the C ABI from pinned HOST
              buffers: mrn_transfer_convert host AoS -> device target for
              every collection, then the status word read back
cpu_baseline  the CPU oracle (plain C) on a bounded sample of the same jobs
batched_vs_per_call  the same jobs with one mrn_convert launch each
extras        single conversions (configs 1-3 and 2^26 scale-ups), the
              transfer chunk sweep against the host link, the 16-collection
              cell batch, the sensor grid, collections, the served sweep

Before timing, a seeded sample of the batch (every tracks job of at most
200,000 parents and every 64th job) is compared byte for byte with the
oracle, and the timed outputs are compared with the checked ones.

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
MIXED_SEED = 3
KERNEL_SOURCES = ["paper_2511_04853_b300/csrc/mrn_kernels.cu", "paper_2511_04853_b300/csrc/mrn_device.cuh",
                  "paper_2511_04853_b300/csrc/mrn_plan.h"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--batch", type=int, default=BATCH, help="collections of the cell batch extra")
    ap.add_argument("--device-only", action="store_true",
                    help="profiling runs: only the timed device step (no e2e, baselines or extras)")
    ap.add_argument("--case", default=None,
                    help="profiling runs: repeat one conversion, e.g. cells:aos:soa:16777216 "
                         "(schema:src[/B]:dst[/B]:records), or one overlapping move, memmove:bytes:shift")
    ap.add_argument("--mixed-jobs", type=int, default=4096, help="collections in the mixed batch")
    ap.add_argument("--mixed-only", action="store_true",
                    help="profiling runs: the mixed batch's check and timed steps only")
    ap.add_argument("--serve-rates", default="0.1,0.25,0.5,0.75,0.9,1.0,1.2",
                    help="served arrival rates as fractions of the measured saturation rate")
    ap.add_argument("--serve-requests", type=int, default=10000, help="requests per served rate")
    ap.add_argument("--serve-seconds", type=float, default=30.0, help="offered time per served rate")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the extras (single conversions, sweeps, cell batch, sensor grid, "
                         "collections, serving)")
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


def cells_workload(batch):
    return ("calorimeter cells: %d collections x 200,000 records (24-byte AoS); per collection AoS->SoA, "
            "SoA->AoSoA(32), AoSoA(32)->AoS" % batch)


def workload_config(jobs, alg_bytes=None, records=None):
    """The step's workload: the mixed batch (the short name first)."""
    c = {"workload": "mixed batch: %d collections, one CUDA graph (k_batch x 2 + k_batch_jag_rest)" % jobs,
         "collections": jobs,
         "sizes": "records round(10^U(3,6)), seed %d" % MIXED_SEED,
         "schemas": "uniform over points (32 B AoS), cells (24 B), tracks (24 B + jagged 8 B children, "
                    "lengths min(Poisson(20), 256))",
         "layouts": "AoS source; target uniform over SoA / AoSoA(32) / AoSoA(128)",
         "l2": "inputs larger than L2 (every step streams the whole batch from HBM; L2 126 MB)",
         "parallelism": "replicas"}
    if alg_bytes is not None:
        c["algorithmic_bytes_per_step"] = alg_bytes
    if records is not None:
        c["records"] = records
    return c


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples (every 50 ms) while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc, self.lines = index, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def wait_first(self, timeout=3.0):
        """Waits until nvidia-smi has printed its first sample."""
        t0 = time.time()
        while self.proc is not None and not self.lines and time.time() - t0 < timeout:
            time.sleep(0.01)

    def stop(self, window=None):
        """Median SM clock and the throttle reasons of the samples taken in
        `window` (host times (t0, t1); all samples when None)."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for t, ln in self.lines:
            if window and not (window[0] <= t <= window[1]):
                continue
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

PACKED = {"points": 25, "cells": 24}


def mixed_alg_bytes(name, n, m=0):
    """Algorithmic bytes of one job of the mixed batch: each record read
    once and written once (the packed field bytes on the field-major side);
    tracks: 24 B parent + 8 B per child read, 12 B parent columns + 4 B
    offset + 8 B per child written, plus the last offset."""
    if name == "tracks":
        return 24 * n + 8 * m + 12 * n + 4 * (n + 1) + 8 * m
    return n * ({"points": 32, "cells": 24}[name] + PACKED[name])


def oracle_mixed_sample(stride, jobs=4096, offset=0):
    """Jobs offset, offset + stride, ... of the mixed batch's plan, generated
    on the host by the seeded generator and laid out as AoS by the oracle;
    returns a step that converts every sampled job with the oracle, its
    algorithmic bytes and a description."""
    import datagen
    import oracle
    plan = mixed_plan(jobs)
    schemas = {k: oracle.Schema(datagen.WORKLOAD_SCHEMAS[k]) for k in MIXED_SCHEMAS}
    work, alg = [], 0
    for i in range(offset, len(plan), stride):
        name, n, (dk, db) = plan[i]
        o = schemas[name]
        d = datagen.workload(name, n, 1000 + i)
        src = oracle.pack(o, d, "aos")
        m = d["m"] if name == "tracks" else 0
        work.append((o, src, oracle.alloc(o, dk, n, m, db)))
        alg += mixed_alg_bytes(name, n, m)

    def step():
        for o, src, dst in work:
            st, _ = oracle.convert_into(o, src, dst)
            assert st == 0
    return step, alg, "%d of the %d mixed-batch collections (every %d-th from %d), %.2f GB algorithmic" % (
        len(work), jobs, stride, offset, alg / 1e9)


def cpu_oracle_rate(seconds, stride=64):
    """The oracle (plain C, one thread) on a sample of the mixed batch,
    repeated for about `seconds`; GB/s."""
    step, alg, what = oracle_mixed_sample(stride)
    reps, t0 = 0, time.perf_counter()
    while True:
        step()
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return alg * reps / el / 1e9, reps, el, what


def _oracle_worker(job):
    """One host process of the all-cores oracle measurement: its own slice
    of the sample, the conversions repeated for `seconds` from a common
    start time."""
    seconds, stride, offset, start_at = job
    step, alg, _ = oracle_mixed_sample(stride, offset=offset)
    step()
    while time.time() < start_at:
        time.sleep(0.01)
    reps, t0 = 0, time.perf_counter()
    while True:
        step()
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            return reps * alg, el


def cpu_oracle_rate_all_cores(seconds):
    """The same oracle, unchanged, in one process per host core (spawned:
    the parent already holds a CUDA context), each on its own slice of the
    mixed batch (every 256th job from a per-core offset), all started
    together; aggregate GB/s."""
    import multiprocessing as mp
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    lead = 10.0 + 0.1 * cores
    start_at = time.time() + lead
    pool = ctx.Pool(cores)
    try:
        job = pool.map_async(_oracle_worker, [(seconds, 256, (7 * i) % 256, start_at) for i in range(cores)])
        res = job.get(timeout=lead + seconds + 180.0)  # a worker that died must not hang the bench
    except Exception as e:
        pool.terminate()
        return None, "not measured: %s" % type(e).__name__
    pool.close()
    pool.join()
    return sum(b / el for b, el in res) / 1e9, cores


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle on the step's workload (the mixed
    batch), each step a bounded sample of its collections sized so the
    whole run takes about a minute."""
    if rank != 0:
        return
    probe_step, probe_alg, _ = oracle_mixed_sample(256, args.mixed_jobs)
    t0 = time.perf_counter()
    probe_step()
    rate = probe_alg / max(1e-6, time.perf_counter() - t0)
    per_step_s = 60.0 / max(1, args.steps + args.warmup)
    full = sum(mixed_alg_bytes(nm, n, 20 * n if nm == "tracks" else 0) for nm, n, _ in mixed_plan(args.mixed_jobs))
    stride = int(min(args.mixed_jobs, max(1, full / max(1.0, per_step_s * rate))))
    step, alg, what = oracle_mixed_sample(stride, args.mixed_jobs)
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t0
    val = args.steps * alg / el / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(val, 3), "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(el / args.steps * 1e3, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": workload_config(args.mixed_jobs),
            "cpu_baseline": {"value": round(val, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": "per step: " + what},
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


def build_mixed(mrn, torch, jobs):
    """The mixed batch's collections on the device: AoS sources generated
    with the workload distributions, garbage-filled destinations, and the
    job list (schema name, records, children, target, buffers)."""
    import datagen
    plan = mixed_plan(jobs)
    schemas = {k: mrn.Schema(datagen.WORKLOAD_SCHEMAS[k]) for k in MIXED_SCHEMAS}
    items, alg, alg_jag, parents = [], 0, 0, 0
    t0 = time.perf_counter()
    for i, (name, n, (dk, db)) in enumerate(plan):
        s = schemas[name]
        rec, pool, m = device_aos(torch, s, name, n, 1000 + i)
        out = torch.full((s.required_bytes(dk, n, m, db),), 0xA5, dtype=torch.uint8, device="cuda")
        src = mrn.View(s, "aos", n, base=rec, child_pool=pool, m=m)
        dst = mrn.View(s, dk, n, block=db, base=out, m=m)
        items.append({"name": name, "n": n, "m": m, "dk": dk, "db": db, "rec": rec, "pool": pool,
                      "out": out, "src": src, "dst": dst, "s": s})
        a = mixed_alg_bytes(name, n, m)
        alg += a
        if name == "tracks":
            alg_jag += a
            parents += n
    torch.cuda.synchronize()
    # k_batch (two launches) moves every algorithmic byte
    return {"items": items, "alg": alg, "alg_jag": alg_jag, "alg_plain": alg - alg_jag,
            "parents": parents, "alg_kbatch": alg,
            "records": sum(n for _, n, _ in plan), "setup_s": round(time.perf_counter() - t0, 1),
            "pairs": [(it["src"], it["dst"]) for it in items]}


def oracle_check_mixed(torch, M, max_tracks=200_000, every=64):
    """Compares a seeded sample of the batch's outputs byte for byte with
    the oracle run on the same input bytes: every tracks job of at most
    max_tracks parents and every `every`-th job.  The oracle (a C library
    called through ctypes, which releases the GIL) runs on one thread per
    host core."""
    import numpy as np
    import datagen
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    schemas = {k: oracle.Schema(datagen.WORKLOAD_SCHEMAS[k]) for k in MIXED_SCHEMAS}
    pick = [i for i, it in enumerate(M["items"])
            if (it["name"] == "tracks" and it["n"] <= max_tracks) or i % every == 0]

    def one(i):
        it = M["items"][i]
        o, n, m = schemas[it["name"]], it["n"], it["m"]
        rec = it["rec"][: n * o.stride].cpu().numpy()
        pool = it["pool"][: m * 8].cpu().numpy() if it["pool"] is not None else None
        src = oracle.Side(oracle.AOS, n, m, base=rec, pool=pool)
        dst = oracle.alloc(o, it["dk"], n, m, it["db"])
        st, _ = oracle.convert_into(o, src, dst)
        nb = o.base_bytes(it["dk"], it["db"], n, m)
        got = it["out"][:nb].cpu().numpy()
        return st == 0 and np.array_equal(got, dst.base[:nb]), nb
    t0 = time.perf_counter()
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    with ThreadPoolExecutor(max(1, cores)) as ex:
        res = list(ex.map(one, pick))
    bad = [pick[k] for k, (ok, _) in enumerate(res) if not ok]
    assert not bad, "mixed-batch jobs differ from the oracle: %s" % bad[:10]
    return {"jobs_checked": len(pick), "tracks_jobs_checked": sum(1 for i in pick if M["items"][i]["name"] == "tracks"),
            "output_bytes_compared": int(sum(nb for _, nb in res)), "seconds": round(time.perf_counter() - t0, 1),
            "rule": "every tracks job of <= %d parents and every %d-th job, oracle on the same input bytes, "
                    "bit-exact" % (max_tracks, every)}


def outputs_equal(torch, M, want):
    for k, (it, w) in enumerate(zip(M["items"], want)):
        if not torch.equal(it["out"], w):
            return k
    return -1


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


def traffic_record(kernel):
    """DRAM bytes per algorithmic byte of `kernel` from the committed ncu
    summary, while the kernel sources are the ones it was taken on."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        j = json.load(f)
    if j.get("kernel_source_hash") != kernel_hash():
        return None
    return j.get("kernels", {}).get(kernel)


def roof(alg, ms, peak, peak_src, kernel, ratio_rec, **kw):
    achieved = alg / (ms * 1e-3) / 1e9
    r = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
         "frac": round(achieved / peak, 4),
         "traffic": int(ratio_rec["traffic_per_algorithmic_byte"] * alg) if ratio_rec else None,
         "kernel": kernel, "algorithmic_bytes_per_launch": alg, "launch_ms_mean": round(ms, 5),
         "peak_source": ("of measured (MEASURED_PEAKS.json hbm_gbs, copy read+write)" if peak_src == "measured"
                         else "of fallback 6.4 TB/s")}
    if ratio_rec:
        r["traffic_source"] = "ncu dram__bytes read+write per algorithmic byte on %s, scaled to this launch" % (
            ratio_rec["workload"])
    r.update(kw)
    return r


def timed_steps(mrn, torch, stream, batch, steps, warmup, world, local):
    """Warm-up replays, then `steps` timed replays of the batch's graph with
    events between its kernels in every replay; clocks sampled meanwhile."""
    import torch.distributed as dist
    clk = ClockSampler(local)
    clk.start()
    clk.wait_first()
    for _ in range(warmup):
        batch.launch()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    for e in ev:  # create the events before the timed region
        for x in e:
            x.record(stream)
    torch.cuda.synchronize()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h0 = time.time()
    t_start.record(stream)
    for k in range(steps):
        batch.launch_timed(*ev[k], stream=stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    h1 = time.time()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    time.sleep(0.06)
    clocks = clk.stop(window=(h0, h1))
    clocks["window_s"] = round(h1 - h0, 3)
    total = t_start.elapsed_time(t_end)
    # ev: before the scratch reset, before the first k_batch launch, after
    # k_batch_jag_rest
    return {"ms_per_step": total / steps, "setup": [a.elapsed_time(b) for a, b, _ in ev],
            "k_batch": [b.elapsed_time(c) for _, b, c in ev], "launch": [a.elapsed_time(c) for a, _, c in ev],
            "clocks": clocks}


def run_mine(args, rank, world):
    import torch
    import torch.distributed as dist
    import paper_2511_04853_b300 as mrn
    import datagen

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    peak, peak_src = peaks()
    M = build_mixed(mrn, torch, args.mixed_jobs)
    # autotuner: per-pair tile shapes, then the batch's launch shape
    tuned = {}
    profiling = args.device_only or args.mixed_only
    for name in () if profiling else ("points", "cells"):
        s = mrn.Schema(datagen.WORKLOAD_SCHEMAS[name])
        for dk, db in MIXED_TARGETS:
            # tuned on 2^25 records (1.0-1.3 GB per pair, eight times the L2 or
            # more): the batch streams every job from HBM, and at a few times
            # the L2 the direct path wins on cache hits it will not get here
            r = mrn.autotune(s, "aos", dk, 1 << 25, 0, db)
            tuned["%s_aos_to_%s%s" % (name, dk, db or "")] = {k: r[k] for k in ("staged", "threads",
                                                                               "tile_records", "ctas_per_sm")}
    batch = mrn.Batch(M["pairs"], use_graph=True)
    launch_shape = {} if profiling else batch.tune()
    # the measured path is checked before it is timed: a sample against the
    # oracle, then the whole output kept for the checks after timing
    for it in M["items"]:
        it["out"].fill_(0xA5)
    batch.launch()
    assert mrn.sync() == mrn.OK
    parity = oracle_check_mixed(torch, M) if rank == 0 else None
    want = [it["out"].clone() for it in M["items"]]
    T = timed_steps(mrn, torch, stream, batch, args.steps, args.warmup, world, local)
    ms_step = T["ms_per_step"]
    if world > 1:
        t = torch.tensor([ms_step], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    value = world * M["alg"] / (ms_step * 1e-3) / 1e9
    assert mrn.sync() == mrn.OK
    bad = outputs_equal(torch, M, want)
    assert bad < 0, "timed output of job %d differs from the checked output" % bad
    lm, lj, lb = (statistics.mean(T[k]) for k in ("launch", "setup", "k_batch"))
    ntr = sum(1 for it in M["items"] if it["name"] == "tracks")
    roofline = roof(M["alg_kbatch"], lb, peak, peak_src, "k_batch (the %d points / cells jobs, and the %d tracks "
                    "jobs' parents with their offsets and child pools; persistent)" % (len(M["items"]) - ntr, ntr),
                    traffic_record("k_batch"),
                    launch_samples="every timed replay (%d), events recorded inside the graph" % args.steps,
                    step={"launch_ms_mean": round(lm, 5), "ms_per_step": round(ms_step, 5),
                          "gbps": round(M["alg"] / (lm * 1e-3) / 1e9, 1),
                          "frac": round(M["alg"] / (lm * 1e-3) / 1e9 / peak, 4)},
                    per_kernel={"setup": {"ms_mean": round(lj, 4), "algorithmic_bytes": 0,
                                          "what": "the scratch-reset memset node (and the fused jagged launch, "
                                                  "which has no jobs here: every tracks pool fits its "
                                                  "destination)"},
                                "k_batch": {"ms_mean": round(lb, 4), "algorithmic_bytes": M["alg_kbatch"],
                                            "gbps": round(M["alg_kbatch"] / (lb * 1e-3) / 1e9, 1),
                                            "frac": round(M["alg_kbatch"] / (lb * 1e-3) / 1e9 / peak, 4),
                                            "what": "points and cells jobs, tracks parents and offsets, tracks "
                                                    "child pools (16 B per child)",
                                            "note": "both persistent launches (%d parents checked record by "
                                                    "record), and k_batch_jag_rest after them (returns at "
                                                    "once: every pool is canonical)" % M["parents"]}})
    if rank == 0:
        print("step: %.3f ms, %.1f GB/s; k_batch %.3f ms, setup %.3f ms; parity %s" % (
            ms_step, value, lb, lj, parity), file=sys.stderr, flush=True)
    if profiling:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
                              "mode": "device-only (profiling)", "roofline": roofline,
                              "config": workload_config(args.mixed_jobs, M["alg"], M["records"])}), flush=True)
        return
    finish_mine(mrn, torch, stream, args, rank, world, M, batch, want, T, ms_step, value, roofline, parity,
                launch_shape, tuned, peak)


def finish_mine(mrn, torch, stream, args, rank, world, M, batch, want, T, ms_step, value, roofline, parity,
                launch_shape, tuned, peak):
    """Everything after the timed step: the per-call baseline and the
    default-shape batch, e2e, the extras, the CPU baseline, the JSON line."""
    extra = {}
    alg_step, records = M["alg"], M["records"]
    if rank == 0:
        def timed(fn, reps):
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
        # one mrn_convert launch per collection, same kernels, same stream
        for it in M["items"]:
            it["out"].fill_(0xA5)
        per_ms = timed(batch.launch_per_job, 3)
        bad = outputs_equal(torch, M, want)
        assert bad < 0, "per-call output of job %d differs" % bad
        extra["batched_vs_per_call"] = {"per_call_ms_per_step": round(per_ms, 3), "batched_ms_per_step":
                                        round(ms_step, 3), "speedup": round(per_ms / ms_step, 3),
                                        "per_call_launches_per_step": len(M["items"]),
                                        "per_call_gbps": round(M["alg"] / (per_ms * 1e-3) / 1e9, 1)}
        # the autotuner off: default tile shapes and launch shape
        mrn.autotune_clear()
        plain = mrn.Batch(M["pairs"], use_graph=True)
        for it in M["items"]:
            it["out"].fill_(0xA5)
        def_ms = timed(plain.launch, 5)
        bad = outputs_equal(torch, M, want)
        assert bad < 0, "default-shape output of job %d differs" % bad
        del plain
        extra["autotuner"] = {"default_shapes_ms_per_step": round(def_ms, 3), "autotuned_ms_per_step":
                              round(ms_step, 3), "gain": round(def_ms / ms_step, 4),
                              "launch_shape": dict(launch_shape, chosen_by="mrn_batch_tune"),
                              "launch_shape_spread": {
                                  "candidates": launch_shape.get("candidates"),
                                  "best_ms": round(launch_shape.get("ms", 0.0), 3),
                                  "worst_ms": round(launch_shape.get("worst_ms", 0.0), 3),
                                  "worst_over_best": round(launch_shape.get("worst_ms", 0.0)
                                                           / max(1e-9, launch_shape.get("ms", 1.0)), 4),
                                  "space": "chunk {1,2,4,8,16} x CTAs per SM {occupancy, 2} for both "
                                           "k_batch launches"},
                              "pair_shapes": tuned}
    link = host_link(torch, stream) if rank == 0 else None
    e2e = run_e2e_mixed(mrn, torch, M, world, link, want)
    del batch, want
    for it in M["items"]:
        it["out"] = None
    M.clear()
    torch.cuda.empty_cache()
    if rank != 0:
        return
    if not args.no_extras:
        extra["host_link_gbps"] = link
        extra.update(secondary(mrn, torch, stream, peak, link))
        extra["cells_batch_16x3"] = run_cells_batch(mrn, torch, stream, peak, args)
        extra["sensor_grid"] = run_sensor_grid(mrn, torch, stream)
        extra["collection_ops"] = run_collection_ops(mrn, torch, stream, peak)
        extra["served"] = run_served(mrn, torch, args)
    cpu_val, cpu_reps, cpu_s, cpu_what = cpu_oracle_rate(10.0)
    cpu_all, cpu_cores = cpu_oracle_rate_all_cores(10.0)
    line = {"metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic (seeded generators; distributions of the points / cells / tracks workloads)",
            "config": workload_config(args.mixed_jobs, alg_step, records),
            "e2e": e2e, "gpu_launches": 3 * args.steps, "roofline": roofline,
            "cpu_baseline": {"value": round(cpu_val, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": "%s, converted %d times (%.1f s)" % (cpu_what, cpu_reps, cpu_s),
                             "all_cores": {"value": round(cpu_all, 3) if cpu_all else None, "unit": "GB/s",
                                           "cores": cpu_cores,
                                           "sample": "one process per core, each every 256th collection from "
                                                     "its own offset, 10 s, started together; aggregate"}},
            "clocks": T["clocks"]}
    # the large extras first, the headline's own evidence last (the tail of
    # a long line is what survives truncation)
    for k in ("served", "collection_ops", "sensor_grid", "single_collection", "cells_batch_16x3"):
        if k in extra:
            line[k] = extra.pop(k)
    line.update(extra)
    line["parity_sample"] = parity
    print(json.dumps(line), flush=True)


def host_link(torch, stream):
    """Pinned host <-> device copies of 1 GiB (best of 5) and both
    directions at once: the bound of every transfer path."""
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
    out = {"h2d": round((1 << 30) / (best_h2d * 1e-3) / 1e9, 1),
           "d2h": round((1 << 30) / (best_d2h * 1e-3) / 1e9, 1),
           "both_directions_total": round(2 * (1 << 30) / best_bi / 1e9, 1)}
    del h, h2, dbuf, dbuf2
    torch.cuda.empty_cache()
    return out


def secondary(mrn, torch, stream, peak, link):
    """Single-collection launches at the workload sizes and scale-up
    collections (2^26 records), L2 flushed before each launch, against the
    HBM roofline (small collections also back to back); the transfer chunk
    sweep and the zero-copy ablation against the host link."""
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

    def back_to_back(src, dst, reps=50):
        mrn.convert(src, dst)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            mrn.convert(src, dst)
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / reps

    def row(alg, med, fastest, b2b=None):
        r = {"us_median": round(med * 1e3, 2), "gbps": round(alg / (med * 1e-3) / 1e9, 1),
             "frac_of_hbm": round(alg / (med * 1e-3) / 1e9 / peak, 3),
             "gbps_mean_fastest_fifth": round(alg / (statistics.mean(fastest) * 1e-3) / 1e9, 1),
             "algorithmic_bytes": alg}
        if b2b is not None:
            r["us_back_to_back"] = round(b2b * 1e3, 2)
        return r

    packed = {"points": 25, "cells": 24}
    rows = {}
    for name, n, pairs in [("points", 10000, [("aos", 0, "soa", 0), ("soa", 0, "aos", 0)]),
                           ("cells", 200000, [("aos", 0, "soa", 0), ("soa", 0, "aosoa", 32),
                                              ("aosoa", 32, "aos", 0)]),
                           ("cells", 1 << 26, [("aos", 0, "soa", 0), ("soa", 0, "aos", 0),
                                               ("soa", 0, "aosoa", 32), ("aosoa", 32, "aos", 0)]),
                           ("points", 1 << 26, [("aos", 0, "soa", 0), ("soa", 0, "aos", 0),
                                                ("aosoa", 32, "aos", 0)])]:
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
            b2b = back_to_back(src, dst) if n < 1e6 else None
            key = "%s_%d_%s%s_to_%s%s" % (name, n, sk, sb or "", dk, db or "")
            rows[key] = row(n * (s.stride + packed[name]), med, fastest, b2b)
        del bufs
    # jagged tracks, AoS -> SoA and back (canonical child pool)
    s = mrn.Schema(datagen.TRACKS)
    for n in (100000, 1 << 22):
        m, recs, pool = jagged_aos(torch, s, n)
        soa = torch.empty(s.required_bytes("soa", n, m), dtype=torch.uint8, device="cuda")
        src = mrn.View(s, "aos", n, base=recs, child_pool=pool, m=m)
        dst = mrn.View(s, "soa", n, base=soa, m=m)
        alg = mixed_alg_bytes("tracks", n, m)
        med, fastest = time_conv(src, dst, 10)
        b2b = back_to_back(src, dst) if n < 1e6 else None
        rows["tracks_%d_aos_to_soa" % n] = dict(row(alg, med, fastest, b2b), children=m)
        back = mrn.View(s, "aos", n, base=recs, child_pool=pool, m=m)
        med, fastest = time_conv(dst, back, 10)
        b2b = back_to_back(dst, back) if n < 1e6 else None
        rows["tracks_%d_soa_to_aos" % n] = row(alg, med, fastest, b2b)
        assert mrn.sync() == mrn.OK
        del recs, pool, soa
    # the points record with its position as one interleaved f32[3] array
    s = mrn.Schema(datagen.POINTS_INTERLEAVED)
    n = 1 << 26
    bufs = {}
    for k, bk in (("aos", 0), ("soa", 0), ("aosoa", 32)):
        bufs[(k, bk)] = torch.full((s.required_bytes(k, n, 0, bk),), 0x3C, dtype=torch.uint8, device="cuda")
    for sk, sb, dk, db in (("aos", 0, "soa", 0), ("soa", 0, "aos", 0), ("aos", 0, "aosoa", 32),
                           ("aosoa", 32, "aos", 0)):
        src = mrn.View(s, sk, n, block=sb, base=bufs[(sk, sb)])
        dst = mrn.View(s, dk, n, block=db, base=bufs[(dk, db)])
        med, fastest = time_conv(src, dst, 10)
        rows["points_interleaved_%d_%s%s_to_%s%s" % (n, sk, sb or "", dk, db or "")] = row(n * (32 + 25), med,
                                                                                          fastest)
    assert mrn.sync() == mrn.OK
    del bufs
    # nested jagged tracks (hits with samples), canonical pools
    s = mrn.Schema(datagen.TRACKS_NESTED)
    n = 1 << 21
    m, m2, recs, pool, gpool = nested_aos(torch, s, n)
    alg = nested_alg_bytes(n, m, m2)
    a_view = mrn.View(s, "aos", n, base=recs, child_pool=pool, m=m, m2=m2, grandchild_pool=gpool)
    for kind, blk in (("soa", 0), ("aosoa", 32)):
        fm = torch.empty(s.required_bytes_nested(kind, n, m, m2, blk), dtype=torch.uint8, device="cuda")
        f_view = mrn.View(s, kind, n, block=blk, base=fm, m=m, m2=m2)
        med, fastest = time_conv(a_view, f_view, 10)
        rows["tracks_nested_%d_aos_to_%s%s" % (n, kind, blk or "")] = dict(row(alg, med, fastest), children=m,
                                                                            grandchildren=m2)
        back = mrn.View(s, "aos", n, base=recs, child_pool=pool, m=m, m2=m2, grandchild_pool=gpool)
        med, fastest = time_conv(f_view, back, 10)
        rows["tracks_nested_%d_%s%s_to_aos" % (n, kind, blk or "")] = row(alg, med, fastest)
        assert mrn.sync() == mrn.OK
        del fm
    del recs, pool, gpool
    rows["bytes_rule"] = ("algorithmic bytes: points 32 + 25 B/record (interleaved too), cells 24 + 24 B/record, "
                          "tracks 40 + 16 x length B/parent (+4 B for the last offset), nested tracks "
                          "40 B/parent + 36 B/hit + 8 B/sample (+8 B for the last offsets)")
    out["single_collection"] = rows
    del flush
    out["transfer_chunk_sweep"] = chunk_sweep(mrn, torch, stream, link)
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
    torch.cuda.empty_cache()
    return out


def chunk_sweep(mrn, torch, stream, link):
    """Host pinned AoS <-> device SoA for the 200,000-record cell collection
    (4.8 MB of source) at chunk sizes 64 KiB ... 16 MiB, against a plain
    pinned copy of the same bytes timed the same way (the control) and the
    1 GiB host link; source bytes per second, mean over 30 calls."""
    import datagen
    n = 200000
    s = mrn.Schema(datagen.CELLS)
    h_aos = torch.full((n * 24,), 0x3C, dtype=torch.uint8).pin_memory()
    d_soa = torch.empty(s.required_bytes("soa", n), dtype=torch.uint8, device="cuda")
    d_raw = torch.empty(n * 24, dtype=torch.uint8, device="cuda")
    hv = mrn.View(s, "aos", n, base=h_aos, mem="pinned")
    dv = mrn.View(s, "soa", n, base=d_soa)
    reps = 30

    def rate(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        b.synchronize()
        return n * 24 / (a.elapsed_time(b) / reps * 1e-3) / 1e9

    out = {"collection": "cells, 200,000 records, 4.8 MB AoS source", "unit": "GB/s of source bytes",
           "control_pinned_copy": {"h2d": round(rate(lambda: d_raw.copy_(h_aos, non_blocking=True)), 1),
                                   "d2h": round(rate(lambda: h_aos.copy_(d_raw, non_blocking=True)), 1)},
           "points": []}
    for k in range(9):
        chunk = (64 << 10) << k
        h2d = rate(lambda: mrn.transfer_convert(hv, dv, chunk_bytes=chunk, stream=stream))
        d2h = rate(lambda: mrn.transfer_convert(dv, hv, chunk_bytes=chunk, stream=stream))
        p = {"chunk_bytes": chunk, "h2d": round(h2d, 1), "d2h": round(d2h, 1),
             "h2d_frac_of_control": round(h2d / out["control_pinned_copy"]["h2d"], 3),
             "d2h_frac_of_control": round(d2h / out["control_pinned_copy"]["d2h"], 3)}
        if link:
            p["h2d_frac_of_link"] = round(h2d / link["h2d"], 3)
            p["d2h_frac_of_link"] = round(d2h / link["d2h"], 3)
        out["points"].append(p)
    assert mrn.sync() == mrn.OK
    del h_aos, d_soa, d_raw
    return out


def mem_available():
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemAvailable:"):
                    return int(ln.split()[1]) * 1024
    except OSError:
        pass
    return 0


def run_e2e_mixed(mrn, torch, M, world, link, want=None, steps=3, n_streams=2):
    """The mixed batch end to end through the public API from pinned host
    memory: per step, every collection host AoS -> device target with
    mrn_transfer_convert (collection i on stream i % n_streams; each
    direction has one copy pipeline per device), then mrn_sync reads the
    device status word back.  All collections when three times their
    source bytes fit in the host's available memory, else every k-th."""
    items = M["items"]
    need = [it["n"] * it["s"].stride + it["m"] * 8 for it in items]
    avail = mem_available()
    k = 1
    while k < len(items) and 3 * sum(need[::k]) > avail:
        k *= 2
    pick = list(range(0, len(items), k))

    def up(x):
        return (x + 255) // 256 * 256
    total = sum(up(items[i]["n"] * items[i]["s"].stride) + up(items[i]["m"] * 8) for i in pick)
    hbuf = torch.empty(max(1, total), dtype=torch.uint8, pin_memory=True)
    views, pos = [], 0
    for i in pick:
        it = items[i]
        nb = it["n"] * it["s"].stride
        hb = hbuf[pos: pos + nb]
        hb.copy_(it["rec"][:nb])
        pos += up(nb)
        hp = None
        if it["name"] == "tracks":
            pb = hbuf[pos: pos + it["m"] * 8]
            pb.copy_(it["pool"][: it["m"] * 8])
            hp = pb
            pos += up(it["m"] * 8)
        views.append((mrn.View(it["s"], "aos", it["n"], base=hb, child_pool=hp, m=it["m"], mem="pinned"),
                      it["dst"]))
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream() for _ in range(n_streams)]
    main = torch.cuda.current_stream()

    def step():
        for st in streams:
            st.wait_stream(main)
        for j, (hv, dv) in enumerate(views):
            mrn.transfer_convert(hv, dv, stream=streams[j % n_streams])
        for st in streams:
            main.wait_stream(st)
        return mrn.sync(main)

    for i in pick:
        items[i]["out"].fill_(0xA5)
    assert step() == mrn.OK
    if want is not None:
        for i in pick:
            assert torch.equal(items[i]["out"], want[i]), "end-to-end output of job %d differs" % i
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        assert step() == mrn.OK
    el = (time.perf_counter() - t0) / steps
    alg = sum(mixed_alg_bytes(items[i]["name"], items[i]["n"], items[i]["m"]) for i in pick)
    bi = sum(need[i] for i in pick)
    out = {"value": round(world * alg / el / 1e9, 2), "unit": "GB/s", "h2d_bytes_per_step": bi,
           "d2h_bytes_per_step": 4, "ms_per_step": round(el * 1e3, 2), "steps": steps,
           "collections": len(pick), "collections_rule": "all" if k == 1 else "every %d-th (host memory)" % k,
           "path": "mrn_transfer_convert host pinned AoS -> device target (4 MiB chunks, 4 slots; jagged: "
                   "whole source staged), collection i on stream i %% %d, then mrn_sync (4-byte status read)"
                   % n_streams,
           "host_link_gbps": round(bi / el / 1e9, 2)}
    if link:
        out["host_link_frac"] = round(bi / el / 1e9 / link["h2d"], 3)
        out["host_link_measured_h2d_gbps"] = link["h2d"]
    del hbuf, views
    return out


def run_cells_batch(mrn, torch, stream, peak, args):
    """The cell batch: 16 collections of 200,000 cells, each converted
    AoS -> SoA, SoA -> AoSoA(32) and AoSoA(32) -> AoS, 48 conversions in one
    graph replay, against one launch per conversion."""
    import datagen
    s = mrn.Schema(datagen.CELLS)
    colls = make_inputs(mrn, torch, s, args.batch)
    batch = mrn.Batch(pairs_for(mrn, s, colls), use_graph=True)
    shape = batch.tune()
    batch.launch()
    assert mrn.sync() == mrn.OK
    check_outputs(torch, colls)
    step_bytes = args.batch * bytes_per_collection()

    def timed(fn, reps):
        for _ in range(3):
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
    ms = timed(batch.launch, 200)
    check_outputs(torch, colls)
    per = timed(batch.launch_per_job, 20)
    check_outputs(torch, colls)
    del batch, colls
    torch.cuda.empty_cache()
    return {"workload": cells_workload(args.batch), "algorithmic_bytes_per_launch": step_bytes,
            "ms_per_launch_back_to_back": round(ms, 4), "gbps": round(step_bytes / (ms * 1e-3) / 1e9, 1),
            "frac_of_hbm": round(step_bytes / (ms * 1e-3) / 1e9 / peak, 3),
            "per_call_ms": round(per, 4), "speedup_vs_per_call": round(per / ms, 3),
            "launch_shape": shape}


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
    fraction of it is offered for --serve-requests requests or
    --serve-seconds seconds, whichever ends first.  Latency (submission ->
    completion) is reported overall and per decade of request size."""
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

    def pct(v, q):
        v = sorted(v)
        return v[min(len(v) - 1, max(0, int(np.ceil(q * len(v))) - 1))] if v else None

    for frac in [float(x) for x in args.serve_rates.split(",") if x]:
        lam = frac * sat
        sv = mrn.Server(budget, max_slots=8, chunk_bytes=4 << 20)
        nreq = int(min(args.serve_requests, max(50, lam * args.serve_seconds)))
        arrivals = np.cumsum(rng.exponential(1.0 / lam, nreq))
        batch = [make_request() for _ in range(nreq)]
        tickets, late = [], 0.0
        t0 = time.perf_counter()
        for (src, dst, nbytes), ta in zip(batch, arrivals):
            now = time.perf_counter() - t0
            if ta > now:
                time.sleep(ta - now)
            else:
                late = max(late, now - ta)
            rc, t = sv.submit(src, dst)
            if rc == mrn.OK:
                tickets.append((t, nbytes))
        lat_by = {}
        for t, nbytes in tickets:
            st_, lat = sv.wait_latency(t, 600.0)
            assert st_ == mrn.OK
            dec = int(np.floor(np.log10(max(1, nbytes))))
            lat_by.setdefault(dec, []).append(lat)
        el = time.perf_counter() - t0
        stt = sv.stats()
        sv.close()
        decades = {"1e%d-1e%d B" % (d, d + 1): {"requests": len(v), "p50_ms": round(pct(v, 0.5), 3),
                                               "p99_ms": round(pct(v, 0.99), 3)}
                   for d, v in sorted(lat_by.items())}
        rates.append({"frac_of_saturation": frac, "offered_req_per_s": round(lam, 1), "requests": nreq,
                      "offered_s": round(float(arrivals[-1]), 2),
                      "p50_ms": round(stt["p50_ms"], 3), "p99_ms": round(stt["p99_ms"], 3),
                      "max_ms": round(stt["max_ms"], 3),
                      "throughput_source_gbps": round(stt["bytes_in"] / el / 1e9, 2),
                      "completed": stt["completed"], "rejected": stt["rejected"],
                      "peak_device_bytes": stt["peak_device_bytes"],
                      "client_max_lateness_ms": round(late * 1e3, 3), "by_source_size": decades})
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
    schemas = dict(datagen.WORKLOAD_SCHEMAS, **datagen.INTERLEAVED_SCHEMAS, **datagen.NESTED_SCHEMAS)
    s = mrn.Schema(schemas[name])
    if name in datagen.NESTED_SCHEMAS:
        m, m2, aos, pool, gpool = nested_aos(torch, s, n)
        fm = torch.empty(s.required_bytes_nested(dk if sk == "aos" else sk, n, m, m2, db if sk == "aos" else sb),
                         dtype=torch.uint8, device="cuda")
        a_view = mrn.View(s, "aos", n, base=aos, child_pool=pool, m=m, m2=m2, grandchild_pool=gpool)
        f_view = mrn.View(s, dk if sk == "aos" else sk, n, block=db if sk == "aos" else sb, base=fm, m=m, m2=m2)
        src, dst = (a_view, f_view) if sk == "aos" else (f_view, a_view)
        if sk != "aos":
            mrn.convert(a_view, f_view)
        nbytes = nested_alg_bytes(n, m, m2)
    elif s.has_jagged:
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
        nbytes = n * (s.stride + sum(c["size"] for c in s.columns))  # AoS record + packed fields
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


def nested_aos(torch, s, n, seed=5):
    """Nested jagged AoS (tracks with hits with samples) with canonical
    pools: parent lengths min(Poisson(20), 256) from the seeded generator,
    per-hit sample counts min(Poisson(3), 32) drawn on the device; returns
    (children, grandchildren, records, child pool, grandchild pool)."""
    import numpy as np
    import datagen
    import paper_2511_04853_b300 as mrn
    ch = mrn.Schema(datagen.TRACKS_NESTED[3][3])  # the hit record, with its own jagged member
    assert s.stride == 24 and s.info.jag_length_offset == 12 and s.info.jag_begin_offset == 16
    assert ch.stride == 24 and ch.info.jag_length_offset == 8 and ch.info.jag_begin_offset == 16
    d = datagen.workload("tracks", n, seed)
    m = d["m"]
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)

    def records(count, stride, lens, len_off, beg_off):
        r = torch.randint(0, 256, (max(1, count * stride),), dtype=torch.uint8, device="cuda", generator=g)
        rv = r[: count * stride].view(count, stride)
        begs = torch.cumsum(lens.to(torch.int64), 0) - lens.to(torch.int64)
        rv[:, len_off:len_off + 4].copy_(lens.to(torch.int32).view(torch.uint8).view(count, 4))
        rv[:, len_off + 4:beg_off].zero_()  # the padding before the begin
        rv[:, beg_off:beg_off + 8].copy_(begs.view(torch.uint8).view(count, 8))
        return r
    lens = torch.from_numpy(d["lengths"].astype(np.int32)).cuda()
    recs = records(n, 24, lens, 12, 16)
    l1 = torch.poisson(torch.full((max(1, m),), 3.0, device="cuda"), generator=g).clamp_(max=32)[:m].to(torch.int32)
    m2 = int(l1.sum().item())
    pool = records(m, 24, l1, 8, 16)
    gpool = torch.randint(0, 256, (max(1, m2 * 4),), dtype=torch.uint8, device="cuda", generator=g)
    return m, m2, recs, pool, gpool


def nested_alg_bytes(n, m, m2):
    """AoS <-> field-major of the nested tracks: records 24 B per parent and
    per hit and 4 B per sample read; 12 B of parent columns, 8 B of hit
    columns, 4 B of sample columns and one 4-byte offset per parent and per
    hit (plus the last of each level) written."""
    return 24 * n + 24 * m + 4 * m2 + 12 * n + 4 * (n + 1) + 8 * m + 4 * (m + 1) + 4 * m2


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
