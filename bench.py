"""ByteStore on GB300: scan + lookup throughput on the 2^30-row sweep column.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (one "step" = one query through the hot path): a 2^30-row int32
column with values in [0, 2^12) drawn Zipf(s=1.0) (the paper's default domain
and skew, Section 6.1), encoded as PP-VBS; the step scans it with `v < c`
(c picked for 10% selectivity) into a result bit vector and looks up every
matching row to int32. Inputs (the encoded column, ~1.2 GB, larger than the
129 MB L2) are resident in HBM before the timed region; no L2 flush is needed.

Under torchrun (N > 1) the ranks hold row shards of ONE column of N x 2^30 rows,
each encoded against the whole column's dictionary (gathered once over a host
group); the step's one exchange is an all-gather of the ranks' selected-row
counts, whose prefix places each rank's values in the whole column's output
order. The value is the rows of all ranks over the slowest rank's time (weak
scaling).

Beside the step, the line carries two more measurements (skip them with
--no-batched / --no-serving):
  batched: 256 scan+lookup requests over a pool of 32 resident columns
    (2^20..2^28 rows, log-uniform; 8..32-bit codes; Zipf s in [0, 1.5]; all
    three layouts), run as one persistent graph-captured launch vs 256 plain
    scan+lookup launch pairs, with identical outputs checked;
  serving: 16 resident PP-VBS columns (4 tables of 4 columns, 2^28..2^30
    rows), Poisson arrivals at 1k..100k queries/s of 1-3-predicate
    conjunctions + lookup at 0.01%..10% selectivity, through the serving loop
    vs serial plain execution: throughput, p50/p99 latency, identical results.

--impl reference times the CPU oracle (plain C: decode every row from the
layout, evaluate the predicate on the plain value, gather values) on a bounded
sample of the same column on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# side files (clock samples, the batch shape cache): BENCH_OUT_DIR, else the temp dir
OUT_DIR = os.environ.get("BENCH_OUT_DIR") or __import__("tempfile").gettempdir()

METRIC = "scan Grows/s & % of HBM roofline; lookup Gvals/s; batched p50/p99 latency"
WORKLOAD = "sweep column d=12 Zipf s=1.0 PP-VBS, v < c at 10% + lookup"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def profile_traffic(name: str):
    """DRAM bytes per launch of a kernel at the bench's full size, from the
    committed ncu summary profiles/<name>.md (its 'traffic_bytes_full_launch'
    line), or None when the summary is missing or the kernel sources it names
    ('sources' line) no longer hash to its 'sources_sha256' line."""
    import hashlib
    path = os.path.join(ROOT, "profiles", name + ".md")
    if not os.path.exists(path):
        return None
    fields = {}
    with open(path) as f:
        for line in f:
            if ":" in line and line.startswith("- "):
                k, v = line[2:].split(":", 1)
                fields[k.strip()] = v.strip().strip("`")
    try:
        h = hashlib.sha256()
        for src in fields["sources"].split(","):
            with open(os.path.join(ROOT, src.strip()), "rb") as f:
                h.update(f.read())
        if h.hexdigest() != fields["sources_sha256"]:
            return None
        return int(fields["traffic_bytes_full_launch"])
    except (KeyError, OSError, ValueError):
        return None


class Clocks:
    """Samples nvidia-smi every 200 ms while the timed region runs."""

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = os.path.join(OUT_DIR, "clocks_rank%d.csv" % gpu)

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax = float(p[2])
                except ValueError:
                    continue
                for nm, v in zip(names, p[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def _cpulist(text):
    cpus = set()
    for part in text.strip().split(","):
        if not part:
            continue
        a, _, b = part.partition("-")
        cpus.update(range(int(a), int(b or a) + 1))
    return cpus


def bind_near_gpu(local):
    """Restricts this process to the CPUs of the NUMA node its GPU hangs off
    (read from sysfs for the GPU's PCI address), so that pinned host buffers
    allocated afterwards sit in that node's memory; host-to-device traffic then
    avoids the link between CPU sockets. Returns the node, or None when it
    cannot be determined (nothing changed)."""
    try:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")
        sel = vis[local].strip() if local < len(vis) and vis[local].strip() else str(local)
        out = subprocess.run(["nvidia-smi", "-i", sel, "--query-gpu=pci.bus_id", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=30).stdout.strip().splitlines()
        if len(out) != 1:
            return None
        dom, rest = out[0].strip().split(":", 1)
        bdf = "%04x:%s" % (int(dom, 16), rest.lower())
        with open("/sys/bus/pci/devices/%s/numa_node" % bdf) as f:
            node = int(f.read())
        if node < 0:
            return None
        with open("/sys/devices/system/node/node%d/cpulist" % node) as f:
            cpus = _cpulist(f.read()) & os.sched_getaffinity(0)
        if not cpus:
            return None
        os.sched_setaffinity(0, cpus)
        return node
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        return None


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_column(n, seed):
    from paper_2209_00220_gb300 import synth
    values = synth.config_sweep_column(n, 12, 1.0, seed)
    lit, _ = synth.pick_literals(values, "lt", 0.10, seed)
    return values, lit


def shard_column(n_per_rank, world, rank, group=None, seed=0):
    """This rank's row range of ONE column of n_per_rank * world rows (the
    bench column, generated piecewise: row i depends on i alone), the whole
    column's dictionary and counts (all-gathered from the ranks over `group`),
    and the literal (picked on rank 0's rows, shared by all ranks). With one
    rank this is make_column's column and literal."""
    from paper_2209_00220_gb300 import shard, synth
    total = n_per_rank * world
    lo, hi = shard.shard_range(total, world, rank)
    values = synth.config_sweep_column(hi - lo, 12, 1.0, seed, start=lo)
    dictionary = shard.global_dictionary(values, group)
    lit = synth.pick_literals(values, "lt", 0.10, seed)[0] if rank == 0 else 0
    if world > 1:
        import torch.distributed as dist
        box = [lit]
        dist.broadcast_object_list(box, src=0, group=group)
        lit = int(box[0])
    return values, lo, hi, dictionary, int(lit)


def oracle_sample(values, lit, rows, threads=1):
    """Time the oracle pipeline on the first `rows` rows: build the plain PP-VBS
    layout (not timed), then decode every row, scan, look up. With threads > 1
    the rows are split into that many ranges (multiples of 32 rows), each run
    by the oracle's own sequential code on a thread of its own (the oracle's C
    calls release the interpreter lock): the range decoder starts its cursors
    where a full pass has them, and the per-range values are concatenated.
    Returns (Grows/s, values found, seconds, threads used)."""
    from concurrent.futures import ThreadPoolExecutor
    from oracle import oracle as orc
    v = values[:rows]
    ocol = orc.OracleColumn(v, "ppvbs")
    if threads <= 1:
        t0 = time.perf_counter()
        dec = ocol.decode_values()
        bits = orc.scan_values(dec, "lt", lit)
        out = orc.lookup(dec, bits)
        dt = time.perf_counter() - t0
        return rows / dt / 1e9, int(out.size), dt, 1
    per = ((rows + threads - 1) // threads + 31) // 32 * 32
    ranges = [(a, min(a + per, rows)) for a in range(0, rows, per)]
    ocol.decode_values_range(0, 0)  # prepares the flat layout arrays (not timed)

    def part(r):
        dec = ocol.decode_values_range(r[0], r[1])
        bits = orc.scan_values(dec, "lt", lit)
        return orc.lookup(dec, bits)

    with ThreadPoolExecutor(len(ranges)) as ex:
        t0 = time.perf_counter()
        outs = list(ex.map(part, ranges))
        out = np.concatenate(outs)
        dt = time.perf_counter() - t0
    return rows / dt / 1e9, int(out.size), dt, len(ranges)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


# ------------------------------------------------------------ batched form
def batched_pool(B, seed=0, ncols=32):
    """32 resident columns: lengths log-uniform in [2^20, 2^28], code widths 8..32
    bits, Zipf s uniform in [0, 1.5], layouts PP-VBS / ByteSlice / Bit-Packed in
    turn (fixed-width layouts code value - domain_min over a declared 2^d range)."""
    from paper_2209_00220_gb300 import synth
    r = synth.u64(seed, 4040, 4 * ncols)
    pool = []
    for i in range(ncols):
        logn = 20 + float(r[i] >> np.uint64(11)) / float(1 << 53) * 8
        n = int(2 ** logn)
        d = 8 + int(r[ncols + i] % np.uint64(25))
        s = float(r[2 * ncols + i] % np.uint64(1000)) / 1000 * 1.5
        lay = ("ppvbs", "byteslice", "bitpacked")[i % 3]
        v = synth.config_sweep_column(n, d, s, seed * 1000 + i)
        opts = {} if lay == "ppvbs" else {"domain_bits": d, "domain_min": synth.domain_min_for_bits(d)}
        pool.append((v, B.bs_encode_column(v, lay, **opts), lay, d, s))
    return pool


def batched_requests(pool, nreq=256, seed=0):
    """Per request: a pool column (uniform), an op among <, =, BETWEEN and a
    target selectivity log-uniform in [0.01%, 50%]."""
    from paper_2209_00220_gb300 import synth
    r = synth.u64(seed, 4141, 3 * nreq)
    reqs = []
    for i in range(nreq):
        ci = int(r[i] % np.uint64(len(pool)))
        op = ("lt", "eq", "between")[int(r[nreq + i] % np.uint64(3))]
        tgt = 10 ** (-4 + float(r[2 * nreq + i] >> np.uint64(11)) / float(1 << 53) * np.log10(5000))
        a, b = synth.pick_literals(pool[ci][0], op, tgt, i)
        reqs.append((ci, op, a, b))
    return reqs


def run_batched(B, warmup=2, steps=5, seed=0):
    import torch
    pool = batched_pool(B, seed)
    spec = batched_requests(pool, 256, seed)
    cols = [p[1] for p in pool]
    stream = torch.cuda.current_stream()
    # plain path buffers, and the exact counts from a first plain pass
    bits = {ci: torch.empty(max(1, cols[ci].n_words), dtype=torch.int32, device="cuda") for ci, _, _, _ in spec}
    ws = {ci: torch.empty(B.bs_lookup_workspace_bytes(cols[ci]) // 4 + 1, dtype=torch.int32, device="cuda")
          for ci, _, _, _ in spec}
    cnt = torch.zeros(len(spec), dtype=torch.int64, device="cuda")
    big = torch.empty(max(c.n for c in cols), dtype=torch.int32, device="cuda")
    for i, (ci, op, a, b) in enumerate(spec):
        B.bs_scan(cols[ci], op, a, b, out=bits[ci], stream=stream)
        B.bs_lookup(cols[ci], bits[ci], out=big, count=cnt[i:i + 1], workspace=ws[ci], stream=stream)
    torch.cuda.synchronize()
    counts = cnt.cpu().numpy().astype(np.int64)
    outs_plain = [torch.empty(max(1, int(c)), dtype=torch.int32, device="cuda") for c in counts]
    outs_batch = [torch.empty(max(1, int(c)), dtype=torch.int32, device="cuda") for c in counts]
    cnt_b = torch.zeros(len(spec), dtype=torch.int64, device="cuda")

    def plain_once(evs=None):
        for i, (ci, op, a, b) in enumerate(spec):
            B.bs_scan(cols[ci], op, a, b, out=bits[ci], stream=stream)
            B.bs_lookup(cols[ci], bits[ci], out=outs_plain[i], out_cap=int(counts[i]), count=cnt[i:i + 1],
                        workspace=ws[ci], stream=stream)
            if evs is not None:
                evs[i].record(stream)

    reqs = [{"preds": [(cols[ci], op, a, b)], "out": outs_batch[i], "out_cap": int(counts[i]),
             "count": cnt_b[i:i + 1]} for i, (ci, op, a, b) in enumerate(spec)]
    cache = os.path.join(OUT_DIR, "batch_tune.jsonl")
    os.makedirs(os.path.dirname(cache), exist_ok=True)
    batch = B.bs_batch_create(reqs, autotune=True, tune_cache=cache)
    for _ in range(warmup):
        plain_once()
        batch.launch(stream)
    torch.cuda.synchronize()
    t_plain, t_batch, lat_plain = [], [], []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        evs = [torch.cuda.Event(enable_timing=True) for _ in spec]
        e0.record(stream)
        plain_once(evs)
        torch.cuda.synchronize()
        done = np.array([e0.elapsed_time(e) for e in evs])
        t_plain.append(done[-1])
        lat_plain.append(done)
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        batch.launch(stream)
        b1.record(stream)
        torch.cuda.synchronize()
        t_batch.append(b0.elapsed_time(b1))
    same = bool(torch.equal(cnt, cnt_b)) and all(
        torch.equal(outs_plain[i][:int(counts[i])], outs_batch[i][:int(counts[i])]) for i in range(len(spec)))
    lp = np.concatenate(lat_plain)
    rows = int(sum(cols[ci].n for ci, _, _, _ in spec))
    tb, tp = float(np.median(t_batch)), float(np.median(t_plain))
    return {"requests": len(spec), "columns": len(cols), "pool_rows": int(sum(c.n for c in cols)),
            "rows_scanned": rows, "selected": int(counts.sum()),
            "plain_ms": round(tp, 4), "batched_ms": round(tb, 4), "speedup": round(tp / tb, 3),
            "batched_grows_s": round(rows / (tb / 1e3) / 1e9, 2), "plain_grows_s": round(rows / (tp / 1e3) / 1e9, 2),
            "p50_ms": round(tb, 4), "p99_ms": round(tb, 4),
            "plain_p50_ms": round(float(np.percentile(lp, 50)), 4), "plain_p99_ms": round(float(np.percentile(lp, 99)), 4),
            "latency": "closed loop: all 256 submitted at t=0; a batched request completes with its launch",
            "identical": same, "shape": batch.shape(), "gpu_launches_per_batch": 2}


# ------------------------------------------------------------ serving form
SERVE_LENGTHS = (1 << 28, 1 << 29, 759250125, 1 << 30)  # 2^28, 2^29, 2^29.5, 2^30 rows


def serving_tables(B, seed=0, scale=1.0):
    """16 resident PP-VBS columns as 4 equal-length tables of 4 columns (table
    lengths 2^28 .. 2^30 rows); per column a code width of 10..24 bits and a Zipf
    s in [0, 1.5]. Host values are dropped after encoding; a 2^16-row sample of
    each column stays for picking literals."""
    from concurrent.futures import ThreadPoolExecutor
    from paper_2209_00220_gb300 import synth
    r = synth.u64(seed, 5050, 32)
    tables = []
    for t, n0 in enumerate(SERVE_LENGTHS):
        n = max(1 << 16, int(n0 * scale))

        def gen(j, t=t, n=n):
            i = 4 * t + j
            d = 10 + int(r[i] % np.uint64(15))
            s = float(r[16 + i] % np.uint64(1000)) / 1000 * 1.5
            return synth.config_sweep_column(n, d, s, 7000 + i), d, s

        with ThreadPoolExecutor(4) as ex:
            gen_out = list(ex.map(gen, range(4)))
        cols, samples, meta = [], [], []
        for j, (v, d, s) in enumerate(gen_out):
            idx = (synth.u64(4 * t + j, 98, 1 << 16) % np.uint64(n)).astype(np.int64)
            samples.append(v[idx])
            cols.append(B.bs_encode_column(v, "ppvbs"))
            meta.append((d, round(s, 3)))
        del gen_out
        tables.append((n, cols, samples, meta))
    return tables


def serving_queries(tables, count, seed=0):
    """1-3-predicate conjunctions on the columns of one table (uniform), ops among
    <, =, BETWEEN, >=, overall target selectivity log-uniform in [0.01%, 10%]
    split evenly over the predicates; projection column uniform in the table."""
    from paper_2209_00220_gb300 import synth
    r = synth.u64(seed, 5151, 12 * count)
    out = []
    for i in range(count):
        n, cols, samples, _ = tables[int(r[i] % np.uint64(len(tables)))]
        npred = 1 + int(r[count + i] % np.uint64(3))
        first = int(r[2 * count + i] % np.uint64(4))
        sel = 10 ** (-4 + 3 * float(r[3 * count + i] >> np.uint64(11)) / float(1 << 53))
        preds = []
        for j in range(npred):
            c = (first + j) % 4
            op = ("lt", "eq", "between", "ge")[int(r[(4 + j) * count + i] % np.uint64(4))]
            a, b = synth.pick_literals(samples[c], op, sel ** (1.0 / npred), i * 5 + j)
            preds.append((cols[c], op, a, b))
        proj = cols[int(r[8 * count + i] % np.uint64(4))]
        out.append((preds, proj, n))
    return out


def poisson_arrivals(rate, count, seed):
    from paper_2209_00220_gb300 import synth
    u = (synth.u64(seed, 5252, count) >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    return np.cumsum(-np.log1p(-u) / rate)


def serve_at(B, srv, prepared, arrivals, want_counts):
    """Submits each query at its arrival time; a collector thread waits on the
    tickets in order, records the latency from the scheduled arrival and
    releases the result. Returns (latencies s, completion times s, bad)."""
    import queue
    import threading
    q = queue.Queue()
    lat = np.zeros(len(prepared))
    done_t = np.zeros(len(prepared))
    bad = []

    def collect():
        for _ in range(len(prepared)):
            i, ticket, t_sub = q.get()
            r = srv.wait(ticket, 600000)
            if r["status"] != 0 or (want_counts is not None and r["count"] != want_counts[i]):
                bad.append(i)
            lat[i] = (t_sub - arrivals[i]) + r["latency_us"] * 1e-6
            done_t[i] = t_sub + r["latency_us"] * 1e-6  # seconds after the stream's start
            srv.release(ticket)

    th = threading.Thread(target=collect)
    th.start()
    t0 = time.perf_counter()
    for i, pq in enumerate(prepared):
        due = t0 + arrivals[i]
        while time.perf_counter() < due:
            pass
        t_sub = time.perf_counter()
        q.put((i, srv.submit(pq), t_sub - t0))
    th.join()
    return lat, done_t, bad


def _stream_stats(srv, prepared, arr, counts):
    st0 = srv.stats()
    lat, done_t, bad = serve_at(None, srv, prepared, arr, counts)
    st1 = srv.stats()
    m = len(prepared)
    return {"served_qps": round(m / float(done_t.max()), 1),
            "p50_ms": round(1e3 * float(np.percentile(lat, 50)), 3),
            "p99_ms": round(1e3 * float(np.percentile(lat, 99)), 3),
            "batches": int(st1["batches"] - st0["batches"]),
            "mean_batch": round((st1["completed"] - st0["completed"]) / max(1, st1["batches"] - st0["batches"]), 2),
            "persistent_queries": int(st1["persistent_queries"] - st0["persistent_queries"]),
            "single_query_queries": int(st1["single_query_queries"] - st0["single_query_queries"]),
            "ok": not bad}


def run_serving(B, rates=(1000, 3000, 10000, 30000, 100000), seconds=2.0, max_queries=6000, distinct=1024, scale=1.0,
                seed=0, tables=None, label="resident PP-VBS columns of 2^28..2^30 rows"):
    """Poisson streams of 1-3-predicate conjunction + lookup queries drawn
    (seeded, uniform) from `distinct` generated queries, served twice through
    the same dispatcher and admission: by the batching server (64 queries per
    launch, 2 slots, continuous batching) and by serial plain execution (one
    query per launch, one slot, the single-query kernels). Both are measured
    live: latency from the scheduled arrival to the host seeing the result
    complete. Offered rates: the listed ones and 0.5x, 0.8x and 0.95x the
    batching server's measured capacity (its throughput at the highest rate),
    so that p50 / p99 also describe a steady state below capacity. Every
    count is checked against the serial plain result of the same query, and
    a sample of values against plain bs_scan_conj + bs_lookup calls."""
    import torch
    from paper_2209_00220_gb300 import synth
    t_setup = time.time()
    if tables is None:
        tables = serving_tables(B, seed, scale)
    setup_s = time.time() - t_setup
    distinct_q = serving_queries(tables, distinct, seed)
    max_rows = max(t[0] for t in tables)
    nq = max_queries
    pick = (synth.u64(seed, 5353, nq) % np.uint64(distinct)).astype(np.int64)
    queries = [distinct_q[i] for i in pick]
    torch.cuda.empty_cache()
    budget = dict(result_bytes=16 << 30, scratch_bytes=16 << 30)
    srv = B.bs_server_create(max_batch=64, slots=2, **budget)
    plain = B.bs_server_create(max_batch=1, slots=1, single_query_kernels=True, **budget)
    prepared = [srv.prepare(p, proj) for p, proj, _ in queries]
    # the exact counts of every distinct query, from serial plain execution
    counts_d = np.zeros(distinct, dtype=np.int64)
    tickets = [plain.submit(srv.prepare(p, proj)) for p, proj, _ in distinct_q]
    for i, t in enumerate(tickets):
        r = plain.wait(t, 600000)
        counts_d[i] = r["count"]
        plain.release(t)
    counts = counts_d[pick]
    for s_ in (srv, plain):  # warm-up: the first batches
        warm = [s_.submit(pq) for pq in prepared[:64]]
        for t in warm:
            s_.wait(t, 600000)
            s_.release(t)
    old_si = sys.getswitchinterval()
    sys.setswitchinterval(2e-4)
    runs = []
    try:
        def one(rate, k, sub):
            m = int(min(nq, max(200, rate * seconds)))
            arr = poisson_arrivals(rate, m, seed + k)
            r = {"offered_qps": round(rate, 1), "queries": m}
            if sub:
                r["below_capacity"] = sub
            b = _stream_stats(srv, prepared[:m], arr, counts)
            p = _stream_stats(plain, prepared[:m], arr, counts)
            r.update({k2: v for k2, v in b.items()})
            r.update({"plain_" + k2: v for k2, v in p.items() if k2 in ("served_qps", "p50_ms", "p99_ms", "ok")})
            return r

        for k, rate in enumerate(sorted(rates)):
            runs.append(one(rate, k, None))
        capacity = max(r["served_qps"] for r in runs)
        for k, f in enumerate((0.5, 0.8, 0.95)):
            runs.append(one(f * capacity, 100 + k, f))
    finally:
        sys.setswitchinterval(old_si)
    # exact results: a sample of queries' values, served vs plain calls
    same = True
    bits = torch.empty((max_rows + 31) // 32, dtype=torch.int32, device="cuda")
    for i in range(0, nq, max(1, nq // 24)):
        if counts[i] > (1 << 24):
            continue
        p, proj, _ = queries[i]
        B.bs_scan_conj(p, out=bits)
        v, c = B.bs_lookup(proj, bits, out_cap=int(counts[i]) + 1)
        t = srv.submit(prepared[i])
        r = srv.wait(t, 600000)
        got = srv.values(t, r["count"])
        srv.release(t)
        same = same and int(c.item()) == r["count"] and torch.equal(v[: r["count"]], got)
    srv.destroy()
    plain.destroy()
    rows_in_hbm = sum(4 * t[0] for t in tables)
    return {"workload": label, "columns": sum(len(t[1]) for t in tables),
            "tables": [{"rows": t[0], "cols": t[3]} for t in tables],
            "resident_rows": int(rows_in_hbm // 4), "setup_s": round(setup_s, 1), "distinct_queries": distinct,
            "capacity_qps": capacity, "runs": runs, "identical_values_sample": bool(same),
            "identical_counts": all(r["ok"] and r["plain_ok"] for r in runs),
            "latency": "scheduled Poisson arrival to the host seeing the result complete, both servers live",
            "server": {"max_batch": 64, "slots": 2, "result_bytes": 16 << 30, "scratch_bytes": 16 << 30},
            "plain": {"max_batch": 1, "slots": 1, "single_query_kernels": True}}


def small_serving_tables(B, seed=0):
    """16 resident PP-VBS columns of 2^22..2^24 rows (4 tables of 4), short
    enough that every query runs in the persistent kernel."""
    from paper_2209_00220_gb300 import synth
    r = synth.u64(seed, 5454, 32)
    tables = []
    for t, n in enumerate((1 << 22, 1 << 23, 11863283, 1 << 24)):
        cols, samples, meta = [], [], []
        for j in range(4):
            i = 4 * t + j
            d = 10 + int(r[i] % np.uint64(15))
            s = float(r[16 + i] % np.uint64(1000)) / 1000 * 1.5
            v = synth.config_sweep_column(n, d, s, 9000 + i)
            idx = (synth.u64(i, 97, 1 << 16) % np.uint64(n)).astype(np.int64)
            samples.append(v[idx])
            cols.append(B.bs_encode_column(v, "ppvbs"))
            meta.append((d, round(s, 3)))
        tables.append((n, cols, samples, meta))
    return tables


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    n = 1 << 30
    rows = args.ref_rows
    values, lit = make_column(rows, 0)
    threads = host_cores()
    for _ in range(args.warmup):
        oracle_sample(values, lit, rows, threads)
    times = []
    used = 1
    for _ in range(args.steps):
        g, m, dt, used = oracle_sample(values, lit, rows, threads)
        times.append(dt)
    t = float(np.sum(times))
    value = rows * args.steps / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "Grows/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * t / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "rows": n, "sample_rows": rows},
            "cpu_baseline": {"value": round(value, 6), "unit": "Grows/s", "cores": used, "kind": "oracle",
                             "sample": "first %d rows of the same column, every step, %d threads over row ranges"
                                       % (rows, used)},
            "e2e": {"value": round(value, 6), "unit": "Grows/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _scaled(full_traffic, n):
    """Traffic quoted for the 2^30-row bench column, for the rows actually run."""
    return None if full_traffic is None else int(round(full_traffic * n / float(1 << 30)))


def _timed(stream, fn, steps):
    """Per-step CUDA-event times (ms) of `steps` calls of fn on `stream`."""
    import torch
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    for i in range(steps):
        ev[i].record(stream)
        fn()
    ev[steps].record(stream)
    torch.cuda.synchronize()
    return [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]


def run_ours(args):
    ws, rank, local = _dist()
    numa = bind_near_gpu(local)
    import torch
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2209_00220_gb300 import bytestore as B

    n = args.rows
    if ws > 1:
        # row shards of one column: each rank holds a 2^30-row range, encoded
        # against the whole column's dictionary (gathered over a host group)
        from paper_2209_00220_gb300 import shard
        host_group = dist.new_group(backend="gloo")
        values, lo, hi, dictionary, lit = shard_column(n, ws, rank, host_group)
        t0 = time.time()
        col = shard.encode_shard(B, values, "ppvbs", dictionary, device=local, keep_host=True)
        encode_s = time.time() - t0
        n = hi - lo
        counts_all = torch.zeros(ws, dtype=torch.int64, device="cuda")
    else:
        values, lit = make_column(n, rank)
        t0 = time.time()
        col = B.bs_encode_column(values, "ppvbs", device=local, keep_host=True)
        encode_s = time.time() - t0
    info = col.info()
    nw = col.n_words
    bits = torch.empty(nw, dtype=torch.int32, device="cuda")
    m_est = int(np.count_nonzero(values[: 1 << 22] < lit) / min(n, 1 << 22) * n * 1.05) + 1024
    out = torch.empty(min(n, m_est), dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    fws = torch.empty(B.bs_scan_lookup_workspace_bytes(col) // 4 + 1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    pred = [(col, "lt", lit)]

    ubits = torch.empty_like(bits)
    uout = torch.empty_like(out)
    ucount = torch.zeros_like(count)
    work = torch.empty(B.bs_lookup_workspace_bytes(col) // 4 + 1, dtype=torch.int32, device="cuda")

    # the two implementations of the query: the paper's operators (scan
    # kernel -> result bit vector -> lookup kernels: count, offsets, gather)
    # and the fused kernel (bit vector, values and count in one launch). Each
    # produces the bit vector, the values of the selected rows and their count.
    def unfused(o=None, c=None):
        B.bs_scan(col, "lt", lit, 0, out=ubits, stream=stream)
        B.bs_lookup(col, ubits, out=uout if o is None else o, count=ucount if c is None else c, workspace=work,
                    stream=stream)

    def fused(o=None, c=None):
        B.bs_scan_lookup(pred, out=out if o is None else o, count=count if c is None else c, bits=bits,
                         workspace=fws, stream=stream)

    run = unfused if args.step == "unfused" else fused
    step_count = ucount if args.step == "unfused" else count

    # the step: the query; with row shards also the one exchange of the query
    # path: every rank's count, whose exclusive prefix places its values in the
    # whole column's output order
    def step():
        run()
        if ws > 1:
            dist.all_gather_into_tensor(counts_all, step_count)

    for _ in range(args.warmup):
        unfused()
        fused()
    torch.cuda.synchronize()
    m = int(count.item())
    if m > out.numel():
        out = torch.empty(m, dtype=torch.int32, device="cuda")
        uout = torch.empty(m, dtype=torch.int32, device="cuda")
        for _ in range(2):
            unfused()
            fused()
        torch.cuda.synchronize()

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    clocks = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with clocks:
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for i in range(args.steps):
            ev[i].record(stream)
            step()
        ev[args.steps].record(stream)
        end.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    total_ms = start.elapsed_time(end)
    t = torch.tensor([total_ms], device="cuda")
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())

    # each kernel of both implementations timed alone (CUDA events, same stream)
    scan_ms = _timed(stream, lambda: B.bs_scan(col, "lt", lit, 0, out=ubits, stream=stream), args.steps)
    look_ms = _timed(stream, lambda: B.bs_lookup(col, ubits, out=uout, count=ucount, workspace=work,
                                                   stream=stream), args.steps)
    fused_ms = _timed(stream, fused, args.steps)
    same = int(ucount.item()) == m and int(count.item()) == m and bool(torch.equal(ubits, bits)) and \
        bool(torch.equal(uout[:m], out[:m]))
    h_bits = bits.cpu()

    # end to end through the public API: every step's result (the count and the
    # whole value buffer, copied without a host round trip for the count) lands
    # in pinned host memory; two result buffers alternate so that one step's
    # copy overlaps the next step's kernels
    cap = out.numel()
    outs = [out, uout] if args.step == "fused" else [uout, out]
    cnts = [torch.zeros_like(count), torch.zeros_like(count)]
    h_outs = [torch.empty(cap, dtype=torch.int32, pin_memory=True) for _ in range(2)]
    h_cnts = [torch.empty(1, dtype=torch.int64, pin_memory=True) for _ in range(2)]
    copier = torch.cuda.Stream()
    freed = [None, None]
    e2e_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for i in range(e2e_steps):
        k = i % 2
        if freed[k] is not None:
            stream.wait_event(freed[k])  # buffer k's previous copy is done
        run(outs[k], cnts[k])
        ready = torch.cuda.Event()
        ready.record(stream)
        copier.wait_event(ready)
        with torch.cuda.stream(copier):
            h_cnts[k].copy_(cnts[k], non_blocking=True)
            h_outs[k].copy_(outs[k], non_blocking=True)
        freed[k] = torch.cuda.Event()
        freed[k].record(copier)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - e0) / e2e_steps
    h_cnt = h_cnts[(e2e_steps - 1) % 2]
    e2e_ok = int(h_cnt.item()) == m and bool(torch.equal(h_outs[0][:m], h_outs[1][:m]))

    # correctness of what was timed: the count and a sample of the bit vector
    from oracle import oracle as orc
    samp = slice(0, 1 << 20)
    want = orc.scan_values(values[samp], "lt", lit)
    ok = bool(np.array_equal(h_bits[: want.size].numpy().view(np.uint32), want)) and \
        int(h_cnt.item()) == int(np.count_nonzero(values < lit)) and e2e_ok and same

    hbm, peak_kind = _peaks()
    hb = h_bits.numpy().view(np.uint32)
    fused_bytes = B.bs_scan_lookup_bytes(col, "lt", lit, 0, hb, write_bits=True)["bytes"]
    scan_bytes = B.bs_scan_bytes(col, "lt", lit)["bytes"]
    look_bytes = B.bs_lookup_bytes(col, hb)["bytes"]
    fused_s = float(np.mean(fused_ms)) / 1e3
    scan_s = float(np.mean(scan_ms)) / 1e3
    look_s = float(np.mean(look_ms)) / 1e3
    value = n * ws * args.steps / (total_ms / 1e3) / 1e9

    def roof(name, byts, secs, traffic_name, kernel):
        return {"bound": "hbm", "achieved": round(byts / secs / 1e9, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(byts / secs / 1e9 / hbm, 4), "traffic": _scaled(profile_traffic(traffic_name), n),
                "kernel": kernel, "peak_kind": peak_kind, "algorithmic_bytes": int(byts)}

    r_scan = roof("scan", scan_bytes, scan_s, "scan_dense_ppvbs_sweep", "scan_dense_kernel<PP-VBS>")
    r_look = roof("lookup", look_bytes, look_s, "lookup_ppvbs_k2_sweep",
                  "bs_lookup: lookup_count + lookup_scan + lookup_gather<PP-VBS, K<=2>")
    r_fused = roof("fused", fused_bytes, fused_s, "fused_ppvbs_k2_sweep", "fused_kernel<K<=2, v < c> (bs_scan_lookup)")
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": "Grows/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "rows_per_gpu": n, "selected": m, "selectivity": round(m / n, 5), "K": info["max_code_bytes"],
                   "step": ("bs_scan + bs_lookup: scan kernel, then count, offsets and gather kernels"
                            if args.step == "unfused" else
                            "bs_scan_lookup: result bit vector + values + count in one kernel"),
                   "l2": "inputs larger than L2 (BS_1 = %d MB), no flush" % (n >> 20),
                   "parallelism": ("row shards of one %d-row column (dictionary gathered from the ranks, "
                                   "selected-row counts all-gathered for output offsets)" % (n * ws))
                   if ws > 1 else "single GPU",
                   "host_numa_node": numa},
        "scan_grows_s": round(n / scan_s / 1e9, 3),
        "scan_ms": round(float(np.median(scan_ms)), 4),
        "lookup_gvals_s": round(m / look_s / 1e9, 3),
        "lookup_ms": round(float(np.median(look_ms)), 4),
        # the step's dominant kernel: the lookup (unfused step) or the fused kernel
        "roofline": r_look if args.step == "unfused" else r_fused,
        "roofline_scan": r_scan,
        "fused": {"ms": round(float(np.median(fused_ms)), 4), "grows_s": round(n / fused_s / 1e9, 3),
                  "lookup_gvals_s": round(m / fused_s / 1e9, 3), "identical_to_unfused": same,
                  "roofline": r_fused},
        "unfused": {"ms": round(float(np.median(scan_ms)) + float(np.median(look_ms)), 4),
                    "grows_s": round(n / (scan_s + look_s) / 1e9, 3), "roofline_lookup": r_look},
        "e2e": {"value": round(n / e2e_s / 1e9, 4), "unit": "Grows/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 4 * cap + 8, "steps": e2e_steps,
                "note": "count + value buffer to pinned host memory each step; copies overlap the next step"},
        "gpu_launches": args.steps * (4 if args.step == "unfused" else 1),
        "clocks": clocks.summary(),
        "encode_s": round(encode_s, 2),
        "parity_sample_ok": ok,
    }
    del outs, h_outs, out, uout, ubits, work
    torch.cuda.empty_cache()
    if not args.no_small:
        line["small"] = run_small_block(B)
    if not args.no_sweep_slice:
        torch.cuda.empty_cache()
        line["sweep_d12"] = run_sweep_slice(B, n)
    if not args.no_batched:
        torch.cuda.empty_cache()
        line["batched"] = run_batched(B)
    if not args.no_wide:
        torch.cuda.empty_cache()
        line["wide_table"] = run_wide_table(B)
    if not args.no_serving:
        torch.cuda.empty_cache()
        line["serving"] = run_serving(B, scale=args.serve_scale)
        torch.cuda.empty_cache()
        line["serving_short_columns"] = run_serving(
            B, rates=(1000, 10000, 100000), max_queries=4000, tables=small_serving_tables(B),
            label="resident PP-VBS columns of 2^22..2^24 rows (the persistent kernel serves every query)")
    if rank == 0 and ws == 1 and not args.no_cpu:
        cores = host_cores()
        rows = min(n, args.cpu_rows)
        g_all, _, dt_all, used = oracle_sample(values, lit, rows, cores)
        rows1 = min(n, args.cpu_rows_single)
        g_one, _, dt_one, _ = oracle_sample(values, lit, rows1, 1)
        line["cpu_baseline"] = {"value": round(g_all, 6), "unit": "Grows/s", "cores": used, "kind": "oracle",
                                "sample": "first %d rows of the bench column, decode + scan + lookup on %d threads "
                                          "over row ranges, %.1f s" % (rows, used, dt_all),
                                "host_cores": cores,
                                "single_thread": {"value": round(g_one, 6), "unit": "Grows/s", "cores": 1,
                                                  "sample": "first %d rows, %.1f s" % (rows1, dt_one)}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# ------------------------------------------- the small L2-resident column
def run_small_block(B, warmup=3, steps=20):
    """The 2^20-row single-column case (Zipf 1.0 over 65,536 distinct signed
    int32, v < c at about 10 % + lookup of every match) on PP-VBS and on
    ByteSlice with its declared 16-bit domain. Its 1 MB of BS_1 lives in L2,
    so each call is timed twice: warm (repeated back to back) and with L2
    flushed before every repetition (a 256 MB buffer written in between); no
    HBM roofline is claimed here. Scan, lookup and the fused scan + lookup are
    timed alone; the values are checked against the plain filter."""
    import torch
    from paper_2209_00220_gb300 import synth
    n = 1 << 20
    values, domain = synth.config_single_column(seed=0, n=n)
    lit, _ = synth.pick_literals(values, "lt", 0.10, 0)
    want = values[values < lit]
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {"workload": "single column, 2^20 rows, Zipf 1.0 over 65,536 values, v < c + lookup", "rows": n,
           "selected": int(want.size), "selectivity": round(want.size / n, 5)}
    for lay, opts in (("ppvbs", {}), ("byteslice", {"domain_values": domain})):
        col = B.bs_encode_column(values, lay, **opts)
        bits = torch.empty(col.n_words, dtype=torch.int32, device="cuda")
        out = torch.empty(n, dtype=torch.int32, device="cuda")
        fout = torch.empty(n, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        fcnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        ws = torch.empty(B.bs_lookup_workspace_bytes(col) // 4 + 1, dtype=torch.int32, device="cuda")
        fws = torch.empty(B.bs_scan_lookup_workspace_bytes(col) // 4 + 1, dtype=torch.int32, device="cuda")
        fns = (("scan", lambda: B.bs_scan(col, "lt", lit, out=bits, stream=stream)),
               ("lookup", lambda: B.bs_lookup(col, bits, out=out, count=cnt, workspace=ws, stream=stream)),
               ("fused", lambda: B.bs_scan_lookup([(col, "lt", lit)], out=fout, count=fcnt, workspace=fws,
                                                  stream=stream)))
        r = {}
        for mode in ("warm", "l2_flushed"):
            for name, fn in fns:
                ts = []
                for i in range(warmup + steps):
                    if mode == "l2_flushed":
                        flush.fill_(i & 255)
                    e0.record(stream)
                    fn()
                    e1.record(stream)
                    e1.synchronize()
                    if i >= warmup:
                        ts.append(e0.elapsed_time(e1))
                r["%s_%s_us" % (name, mode)] = round(1e3 * float(np.median(ts)), 2)
        m, fm = int(cnt.item()), int(fcnt.item())
        r["parity"] = bool(m == want.size and fm == want.size and np.array_equal(out[:m].cpu().numpy(), want)
                           and np.array_equal(fout[:fm].cpu().numpy(), want))
        r["scan_grows_s_warm"] = round(n / (r["scan_warm_us"] * 1e3), 2)
        r["lookup_gvals_s_warm"] = round(m / (r["lookup_warm_us"] * 1e3), 2)
        r["fused_grows_s_warm"] = round(n / (r["fused_warm_us"] * 1e3), 2)
        res[lay] = r
        del col
    return res


def run_small(args):
    """--small: the single-column block alone, one JSON line."""
    from paper_2209_00220_gb300 import bytestore as B
    print(json.dumps(run_small_block(B, warmup=args.warmup, steps=args.steps)), flush=True)
    return 0


# ---------------------------------------------- the synthetic wide table
def run_wide_table(B, n=1 << 26, queries=24, seed=6, advise_rows=1 << 22):
    """20 int32 columns (categorical, date-like, a monotone id, heavy-tailed
    amounts, mixed; synth.WIDE_TABLE), each in the layout the advisor's
    deterministic mode picks from its first 2^22 rows; seeded conjunctions of
    1-4 predicates followed by lookups of 2-4 projected columns. Each query runs
    (a) as bs_scan_conj + one bs_lookup per projection and (b) as one fused
    bs_scan_lookup for the first projection (which also writes the bit vector)
    + bs_lookup for the others; both are timed per query (CUDA events) and
    their values compared."""
    import torch
    from paper_2209_00220_gb300 import synth
    names = [w[0] for w in synth.WIDE_TABLE]
    t0 = time.time()
    vals, cols, layouts = [], [], []
    for nm in names:
        v = synth.wide_table_column(nm, n, 1)
        lay = B.bs_advise_layout(v[:advise_rows], B.ADVISE_BYTES_MODEL, host_only=True)["layout"]
        cols.append(B.bs_encode_column(v, lay))
        vals.append(v[:1 << 20].copy())  # a sample for literals
        layouts.append(lay)
        del v
    setup_s = time.time() - t0
    r = synth.u64(seed, 77, 16 * queries)
    stream = torch.cuda.current_stream()
    bits = torch.empty((n + 31) // 32, dtype=torch.int32, device="cuda")
    bits2 = torch.empty_like(bits)
    outs = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(4)]
    outs2 = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(4)]
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    cnt2 = torch.zeros(4, dtype=torch.int64, device="cuda")
    lws = torch.empty(max(B.bs_lookup_workspace_bytes(c) for c in cols) // 4 + 1, dtype=torch.int32, device="cuda")
    fws = torch.empty(max(B.bs_scan_lookup_workspace_bytes(c) for c in cols) // 4 + 1, dtype=torch.int32,
                      device="cuda")
    t_plain, t_fused, same, rows_sel = [], [], True, 0
    for i in range(queries):
        order = synth.permutation(len(names), seed * 1000 + i)
        npred = 1 + int(r[i] % np.uint64(4))
        nproj = 2 + int(r[queries + i] % np.uint64(3))
        preds = []
        for j in range(npred):
            ci = int(order[j])
            op = ("lt", "eq", "between")[int(r[(2 + j) * queries + i] % np.uint64(3))]
            tgt = 10 ** (-2 + 1.8 * float(r[(6 + j) * queries + i] >> np.uint64(11)) / float(1 << 53))
            a, b = synth.pick_literals(vals[ci], op, tgt, seed + i * 4 + j)
            preds.append((cols[ci], op, a, b))
        proj = [cols[int(x)] for x in order[len(names) - nproj:]]

        def plain():
            B.bs_scan_conj(preds, out=bits, stream=stream)
            for k, pc in enumerate(proj):
                B.bs_lookup(pc, bits, out=outs[k], count=cnt[k:k + 1], workspace=lws, stream=stream)

        def fused():
            B.bs_scan_lookup(preds, proj=proj[0], out=outs2[0], count=cnt2[0:1], bits=bits2, workspace=fws,
                             stream=stream)
            for k, pc in enumerate(proj[1:], 1):
                B.bs_lookup(pc, bits2, out=outs2[k], count=cnt2[k:k + 1], workspace=lws, stream=stream)

        plain()
        fused()
        t_plain.append(float(np.median(_timed(stream, plain, 3))))
        t_fused.append(float(np.median(_timed(stream, fused, 3))))
        c = cnt.cpu().numpy()
        rows_sel += int(c[0])
        same = same and bool(torch.equal(cnt[:nproj], cnt2[:nproj])) and bool(torch.equal(bits, bits2)) and all(
            torch.equal(outs[k][:int(c[k])], outs2[k][:int(c[k])]) for k in range(nproj))
    tp, tf = float(np.sum(t_plain)), float(np.sum(t_fused))
    return {"rows": n, "columns": len(names), "layouts": {l: layouts.count(l) for l in set(layouts)},
            "queries": queries, "setup_s": round(setup_s, 1), "selected_rows": rows_sel,
            "plain_ms_total": round(tp, 3), "fused_ms_total": round(tf, 3), "speedup": round(tp / tf, 3),
            "plain_ms_per_query": round(tp / queries, 4), "fused_ms_per_query": round(tf / queries, 4),
            "identical": same}


# --------------------------------------------------- the full layout sweep
SWEEP_WIDTHS = (8, 12, 16, 20, 24, 32)
SWEEP_SKEWS = (0.0, 0.5, 1.0, 1.5)           # 0.0: uniform
SWEEP_OPS = ("lt", "eq", "between")
SWEEP_TARGETS = (0.001, 0.01, 0.1, 0.5, 0.9)


def sweep_points(B, n, widths, skews, hbm, emit=None):
    """Points of the single-column layout sweep on one column length: for each
    code width x value distribution, the column in every layout (fixed-width
    layouts with the declared 2^d range), every predicate and target
    selectivity; scan and lookup each timed alone (CUDA events, median of 5),
    scan bytes from every 16th tile of the host replay (bs_scan_bytes_sampled).
    Returns the points; emit(point) is called for each as it is measured."""
    import torch
    from paper_2209_00220_gb300 import synth
    stream = torch.cuda.current_stream()
    bits = torch.empty((n + 31) // 32, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=5):
        fn()
        ts = []
        for _ in range(reps):
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    points = []
    for d in widths:
        for s in skews:
            v = synth.config_sweep_column(n, d, s, d * 10 + int(s * 2))
            for lay in ("bitpacked", "byteslice", "ppvbs"):
                opts = {} if lay == "ppvbs" else {"domain_bits": d, "domain_min": synth.domain_min_for_bits(d)}
                col = B.bs_encode_column(v, lay, keep_host=True, **opts)
                ws = torch.empty(B.bs_lookup_workspace_bytes(col) // 4 + 1, dtype=torch.int32, device="cuda")
                for op in SWEEP_OPS:
                    for tgt in SWEEP_TARGETS:
                        a, b = synth.pick_literals(v, op, tgt, 7)
                        t_scan = timed(lambda: B.bs_scan(col, op, a, b, out=bits, stream=stream))
                        t_look = timed(lambda: B.bs_lookup(col, bits, out=out, count=cnt, workspace=ws,
                                                           stream=stream))
                        m = int(cnt.item())
                        by = B.bs_scan_bytes(col, op, a, b, stride=16)["bytes"]
                        pt = {"d": d, "s": s, "layout": lay, "op": op, "target": tgt,
                              "selectivity": round(m / n, 5), "scan_ms": round(t_scan, 4),
                              "scan_frac": round(by / (t_scan / 1e3) / 1e9 / hbm, 4),
                              "scan_bytes_per_row": round(by / n, 4), "lookup_ms": round(t_look, 4)}
                        points.append(pt)
                        if emit:
                            emit(pt)
                del col, ws
            del v
    return points


def sweep_summary(points, n):
    out = {}
    for lay in ("ppvbs", "byteslice", "bitpacked"):
        pts = [p for p in points if p["layout"] == lay]
        if not pts:
            continue
        f = np.array([p["scan_frac"] for p in pts])
        out[lay] = {"points": len(pts), "scan_frac_mean": round(float(f.mean()), 4),
                    "scan_frac_median": round(float(np.median(f)), 4),
                    "scan_frac_p10": round(float(np.percentile(f, 10)), 4),
                    "scan_ms_total": round(float(sum(p["scan_ms"] for p in pts)), 2),
                    "lookup_ms_total": round(float(sum(p["lookup_ms"] for p in pts)), 2), "rows": n}
        for op in SWEEP_OPS:
            fo = [p["scan_frac"] for p in pts if p["op"] == op]
            if fo:
                out[lay]["scan_frac_mean_" + op] = round(float(np.mean(fo)), 4)
    return out


def run_sweep(args):
    """--sweep: every point of the layout sweep (every width and distribution),
    one JSON line per point, then one summary line per layout."""
    from paper_2209_00220_gb300 import bytestore as B
    hbm, _ = _peaks()
    pts = sweep_points(B, args.rows, SWEEP_WIDTHS, SWEEP_SKEWS, hbm, emit=lambda p: print(json.dumps(p), flush=True))
    for lay, sm in sweep_summary(pts, args.rows).items():
        print(json.dumps(dict(summary=lay, **sm)), flush=True)
    return 0


def run_sweep_slice(B, n):
    """The sweep's d = 12, Zipf 1.0 column (Section 6.1's defaults) in the
    default line: 3 layouts x {<, =, BETWEEN} x 5 target selectivities."""
    hbm, _ = _peaks()
    pts = sweep_points(B, n, (12,), (1.0,), hbm)
    return {"workload": "layout sweep at d = 12, Zipf s = 1.0, %d rows" % n, "summary": sweep_summary(pts, n),
            "points": [[p["layout"], p["op"], p["target"], p["selectivity"], p["scan_ms"], p["scan_frac"],
                        p["lookup_ms"]] for p in pts],
            "point_fields": ["layout", "op", "target", "selectivity", "scan_ms", "scan_frac", "lookup_ms"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--step", default="unfused", choices=["unfused", "fused"],
                    help="the timed step: scan + lookup kernels (default) or the fused kernel")
    ap.add_argument("--rows", type=int, default=1 << 30)
    ap.add_argument("--ref-rows", type=int, default=1 << 24, help="oracle rows per step of --impl reference")
    ap.add_argument("--cpu-rows", type=int, default=1 << 28, help="oracle rows timed on all host cores")
    ap.add_argument("--cpu-rows-single", type=int, default=1 << 26, help="oracle rows timed on one core")
    ap.add_argument("--no-small", action="store_true", help="skip the 2^20-row single-column block")
    ap.add_argument("--no-wide", action="store_true", help="skip the wide-table block")
    ap.add_argument("--no-sweep-slice", action="store_true", help="skip the d = 12 slice of the layout sweep")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 256-request batched measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serve-scale", type=float, default=1.0, help="serving table lengths x this factor")
    ap.add_argument("--small", action="store_true",
                    help="instead of the step: the 2^20-row L2-resident column, warm and L2-flushed")
    ap.add_argument("--sweep", action="store_true",
                    help="instead of the step: every point of the layout sweep, one JSON line each")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep:
        return run_sweep(args)
    if args.small:
        return run_small(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
