"""Benchmark of the fused query path on GB300.

Default workload: the star join (2^26 fact rows, 4 foreign keys into
dimensions of 2,000 / 30,000 / 200,000 / 2,556 rows, fact clustered by date
with delta-coded date keys), grouped by (dim3 attribute, year), SUM(int64).
One step = one replay of the CUDA graph holding the fused persistent kernel
(chunk scheduling, staging, decode, predicates, probes, aggregation and
result assembly).  The dimension hash builds run once before timing and are
reported separately (``build_ms``).  ``--workload chain`` runs LINEITEM ->
ORDERS -> CUSTOMER: CUSTOMER's table is built by a scan+build kernel,
ORDERS' by a scan+probe+build kernel probing it, and the timed step is the
fused LINEITEM pipeline probing ORDERS' table; each build is timed too
(``chain``).

Prints one JSON line (rank 0): the headline (warm graph replays; cold
replays after an L2 flush reported beside them), the roofline against the
measured copy peak and the 8 TB/s specification, the host-link and device
read peaks (``link_peaks``), the end-to-end host-resident variant, the CPU
oracle at one thread and on every CPU, and, for the default star workload,
the other configurations measured after the headline (``extra``: strings,
all-pass strings, the 64-query batch, a serving sweep).  ``--impl
reference`` times the CPU oracle on a bounded sample of the same workload
instead.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fused rows/s & compressed GB/s vs HBM peak vs unfused chain; p50/p99 query ms"
SPEC_HBM_GBS = 8000.0          # HBM3e bandwidth the GB300 is specified at
L2_BYTES = 128 << 20           # at least the GB300's L2


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001
        return 6800.0, "fallback"


KERNEL_SOURCES = ("fused.cu", "fused_kernel.cuh", "fused_lean.cu", "fused_text.cu", "fused_host.cu", "fused_stage.cu",
                  "fused_wide.cu", "tile.cuh",
                  "dpf_device.cuh", "dpf_internal.h", "kernels.h")


def _code_only(src):
    """C++ source without its comments and blank lines (string and character
    literals kept as they are): what the compiler sees."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            while i < n and src[i] != "\n":
                i += 1
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return "\n".join(line.rstrip() for line in "".join(out).splitlines() if line.strip())


def kernel_source_hash(root=None):
    """Hash of the code (comments and blank lines left out) of the sources
    that define the fused kernel: ties stored ncu counters to the kernel
    build they were taken on."""
    import hashlib
    d = os.path.join(root or ROOT, "paper_2605_10511_gb300", "csrc")
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(d, name), encoding="utf-8") as f:
            h.update(name.encode() + b"\0" + _code_only(f.read()).encode())
    return h.hexdigest()[:16]


def stored_traffic(workload, fact_rows, alg_bytes=None):
    """DRAM bytes per launch of the fused kernel from the committed ncu
    summary of this workload, or None when absent or taken on other kernel
    sources.  A capture of a smaller case is scaled by rows, or (with
    ``alg_bytes``: a batch whose queries differ) by algorithmic bytes."""
    path = os.path.join(ROOT, "profiles", f"fused_kernel_{workload}.txt")
    try:
        kv = {}
        with open(path) as f:
            for line in f:
                if ":" in line and not line.startswith(" "):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("source_hash") != kernel_source_hash():
            return None, "stale (kernel changed since capture)"
        b = float(kv["dram_bytes_per_launch"])
        if alg_bytes is not None:
            a = float(kv["algorithmic_bytes_per_launch"])
            return b * alg_bytes / a, f"ncu capture at {int(a)} algorithmic bytes, scaled by algorithmic bytes"
        rows = float(kv["captured_rows"])
        return b * fact_rows / rows, f"ncu capture at {int(rows)} rows, scaled by rows"
    except Exception:  # noqa: BLE001
        return None, "no capture"


def stored_link_bytes(workload, fact_rows):
    """Bytes the host-resident variant's fused kernel received over the host
    link per launch (ncu ctc__rx_bytes_data_user.sum from the committed
    summary of that capture, scaled by rows), or None when absent or taken
    on other kernel sources."""
    path = os.path.join(ROOT, "profiles", f"fused_kernel_{workload}_host.txt")
    try:
        kv = {}
        with open(path) as f:
            for line in f:
                if ":" in line and not line.startswith(" "):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("source_hash") != kernel_source_hash():
            return None, "stale (kernel changed since capture)"
        rows = float(kv["captured_rows"])
        return float(kv["link_bytes_per_launch"]) * fact_rows / rows, f"ncu capture at {int(rows)} rows, scaled by rows"
    except Exception:  # noqa: BLE001
        return None, "no capture"


def _workload(name, rows):
    import synth
    if name == "star":
        return synth.star_join(rows=rows or (1 << 26), clustered=True)
    if name == "star_unsorted":
        return synth.star_join(rows=rows or (1 << 26), clustered=False)
    if name == "star_year":  # one year of dates on the date-clustered fact (mini block pruning)
        return synth.star_join(rows=rows or (1 << 26), clustered=True, date_year=1994)
    if name == "star_year_unsorted":
        return synth.star_join(rows=rows or (1 << 26), clustered=False, date_year=1994)
    if name == "star_bigint":  # the measure as a BIGINT (FOR64) column
        return synth.star_join(rows=rows or (1 << 26), clustered=True, bigint_measure=True)
    if name == "scan":
        return synth.scan_filter_aggregate(rows=rows or (1 << 20))
    # a join chain LINEITEM -> ORDERS -> CUSTOMER (scan+build, scan+probe+build, fused)
    if name == "chain":
        return synth.chain_join(rows=rows or (1 << 26))
    if name == "chain_sparse":
        return synth.chain_join(rows=rows or (1 << 26), sparse_orderkeys=True)
    if name == "strings":
        return synth.strings(rows=rows or (1 << 25))
    # every row passes (an empty prefix): the group-by takes all 2^25 rows, Zipf-skewed keys
    if name == "strings_all":
        return synth.strings(rows=rows or (1 << 25), prefix=b"")
    # 15 groups, one holding 97 % of the rows: the warp-aggregated group-by
    if name == "groups_hot":
        return synth.hot_groups(rows=rows or (1 << 25))
    # word-based strings, LIKE '%ab%', raw bytes vs FSST
    if name == "strings_text":
        return synth.strings(rows=rows or (1 << 25), text=True, contains=b"ab")
    if name == "strings_fsst":
        return synth.strings(rows=rows or (1 << 25), text=True, contains=b"ab", codec="fsst")
    raise ValueError(name)


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:  # noqa: BLE001
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:  # noqa: BLE001
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def host_cpu():
    """(nproc, CPU model name) of the host running the bench."""
    n = os.cpu_count() or 1
    try:
        n = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        pass
    model = "unknown"
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:  # noqa: BLE001
        pass
    return n, model


def oracle_rows_per_s(w, threads, budget_s=5.0):
    """Times the oracle (as it stands) on a prefix sample of the workload's
    fact table: its pages are encoded first by the oracle's own encoder (the
    loader, untimed), then the query decodes them and evaluates the rows on
    ``threads`` host threads.  The sample grows until one evaluation takes
    about budget_s / 4.  Returns (rows/s, rows, seconds)."""
    import oracle
    n_total = w["tables"][w["fact"]]["rows"]
    rows = min(n_total, 1 << 18)
    while True:
        s = _fact_prefix(w, rows)
        enc = oracle.encode_tables(s)
        t0 = time.perf_counter()
        oracle.run_query(s, encoded=enc, threads=threads)
        dt = time.perf_counter() - t0
        if dt > budget_s / 4 or rows >= n_total:
            return rows / dt, rows, dt
        rows = min(n_total, int(rows * min(8.0, max(2.0, budget_s / 2 / dt))))


def cpu_baselines(w):
    """The oracle on the host cores: every CPU of the process and one thread."""
    n, model = host_cpu()
    rate_all, rows_all, dt_all = oracle_rows_per_s(w, n)
    rate_1, rows_1, dt_1 = oracle_rows_per_s(w, 1)
    return {"value": rate_all, "unit": "rows/s", "cores": n, "kind": "oracle",
            "sample": f"first {rows_all} fact rows, decode + evaluate on {n} threads "
                      f"(pages encoded beforehand, untimed), {dt_all:.2f} s",
            "cpu_model": model, "nproc": n,
            "one_thread": {"value": rate_1, "unit": "rows/s", "cores": 1,
                           "sample": f"first {rows_1} fact rows, decode + evaluate, {dt_1:.2f} s"}}


def time_graph(prep_ctx, prep, stream, torch, steps, warmup, flush=None):
    """CUDA-event time (ms) of each of ``steps`` graph replays of ``prep``
    after ``warmup`` untimed ones; with ``flush`` (a device buffer larger
    than L2) the buffer is rewritten on the stream before every replay, so
    each replay starts with a cold L2 (the write is outside the events)."""
    for _ in range(warmup):
        prep_ctx.launch_graph(prep, stream)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    torch.cuda.synchronize()
    for i in range(steps):
        if flush is not None:
            with torch.cuda.stream(stream):
                flush.fill_(i & 0xff)
        starts[i].record(stream)
        prep_ctx.launch_graph(prep, stream)
        ends[i].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in zip(starts, ends)]


def pcts(per):
    v = sorted(per)

    def q(p):
        return v[min(len(v) - 1, int(round(p / 100 * (len(v) - 1))))]
    return {"p50": q(50), "p90": q(90), "p99": q(99), "mean": statistics.mean(v), "n": len(v)}


def _explicit_tuning(args):
    """True when the command line fixes the launch configuration (or turns
    the autotuner off): the library's defaults fill what it leaves at 0."""
    return bool(args.chunk_rows or args.threads or args.ht != "auto" or args.ctas or args.stage != "default"
                or args.group_agg != "default" or args.no_autotune)


def run_batched(args, dpf, torch, np, local):
    """64 queries of the three shapes over fact tables of log-uniform size
    (2^16..2^26 rows) in ONE persistent launch replayed from a CUDA graph,
    under the launch configuration the library's autotuner picks."""
    import synth
    ws = synth.batched_workloads(n_queries=args.batch_queries, seed=4, max_rows=args.batch_max_rows)
    eng = dpf.Engine(device=local)
    for w in ws:
        eng.load_workload(w)
    stream = torch.cuda.Stream()
    plans = [eng.plan(w, stream) for w in ws]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    best, tune_ms, tuning = None, None, None
    if _explicit_tuning(args):
        tuning = dpf.Tuning(args.chunk_rows, args.threads, dpf.HT_PLACE[args.ht], args.ctas, dpf.STAGING[args.stage],
                            dpf.GROUP_AGG[args.group_agg])
    else:
        best, tune_ms = eng.ctx.autotune(plans, stream, reps=2)
    tune_s = time.perf_counter() - t0
    prep = eng.ctx.prepare(plans, tuning)
    eng.ctx.capture_graph(prep, stream)
    for _ in range(args.warmup):
        eng.ctx.launch_graph(prep, stream)
    first = [eng.ctx.read_result(prep, i) for i in range(len(ws))]
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    for i in range(args.steps):
        starts[i].record(stream)
        eng.ctx.launch_graph(prep, stream)
        ends[i].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    per = sorted(s.elapsed_time(e) for s, e in zip(starts, ends))
    ms_step = starts[0].elapsed_time(ends[-1]) / args.steps
    for i in range(len(ws)):
        assert np.array_equal(eng.ctx.read_result(prep, i), first[i]), "result changed across replays"
    rows = sum(w["tables"][w["fact"]]["rows"] for w in ws)
    alg = sum(eng.fact_bytes(w)[0] for w in ws)
    tuned = eng.ctx.prep_tuning(prep)
    eng.ctx.release(prep)
    # the same 64 queries through the unfused chain, one query at a time
    unf_ms, unf_launches, unf_bytes = 0.0, 0, 0
    if not args.no_unfused:
        for i, w in enumerate(ws):
            r = time_unfused(eng, plans[i], stream, first[i], reps=2, fused_ms=1.0)
            unf_ms += r["ms_per_query"]
            unf_launches += r["launches_per_query"]
            unf_bytes += r["intermediate_bytes"]
    peak, peak_kind = _peaks()
    achieved = alg / (statistics.mean(per) * 1e-3) / 1e9
    traffic, traffic_src = stored_traffic("batched", rows, alg_bytes=alg)
    out = {
        "metric": METRIC, "value": rows / (ms_step * 1e-3), "unit": "rows/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic (seeded; 64 queries of the scan / star / strings shapes)",
        "config": {"workload": f"batched_{len(ws)}_queries", "fact_rows_total": rows,
                   "max_rows_per_query": args.batch_max_rows,
                   "queries": len(ws), "l2": "inputs larger than L2", "tuning": tuned},
        "autotune": {"best": best, "best_ms": tune_ms, "search_s": tune_s},
        "compressed_gbs": achieved, "compressed_bytes": alg,
        "latency_ms": {"p50": per[len(per) // 2], "p99": per[min(len(per) - 1, int(0.99 * (len(per) - 1) + 0.5))]},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "traffic_source": traffic_src,
                     "peak_kind": f"{peak_kind} copy bandwidth (burst)"},
        "unfused": None if args.no_unfused else {
            "ms_per_batch": unf_ms, "launches_per_batch": unf_launches, "intermediate_bytes": unf_bytes,
            "fused_speedup": unf_ms / ms_step},
        "gpu_launches": args.steps, "clocks": clocks,
    }
    eng.close()
    print(json.dumps(out), flush=True)


def serve_sweep(dpf, np, local, rows, placement, rates, seconds, max_queries):
    """Poisson streams of queries at several rates through the
    continuous-batching server over a resident star schema: per rate, p50 /
    p90 / p99 latency (submit to result on the host), achieved QPS and
    throughput; every result is checked against the same query run alone."""
    import synth
    w = synth.star_join(rows=rows, clustered=placement == "device")
    eng = dpf.Engine(device=local)
    try:
        t0 = time.perf_counter()
        eng.load_workload(w, fact_placement=placement)
        load_s = time.perf_counter() - t0
        qs = synth.serve_variants(w, 12, 4, seed=5)
        plans = [eng.plan(v) for v in qs]
        ref = [eng.run(v) for v in qs]  # each query alone
        alg = [eng.fact_bytes(v)[0] for v in qs]
        rng = np.random.default_rng(7)
        lines = []
        for lam in rates:
            n = int(min(max_queries, max(20, lam * seconds)))
            gaps = rng.exponential(1.0 / lam, n)
            pick = rng.integers(0, len(qs), n)
            with dpf.Server(eng.ctx, max_batch=64, max_inflight=2) as srv:
                tickets = []
                t_start = time.perf_counter()
                due = t_start
                for k in range(n):
                    due += gaps[k]
                    while True:
                        d = due - time.perf_counter()
                        if d <= 0:
                            break
                        time.sleep(min(d, 0.002) if d > 0.0005 else 0)
                    tickets.append(srv.submit(plans[pick[k]]))
                lat, batch, mismatch = [], [], 0
                for k, tk in enumerate(tickets):
                    got, tm = srv.wait(tk)
                    mismatch += int(not np.array_equal(got, ref[pick[k]]))
                    lat.append((tm["done_us"] - tm["submit_us"]) / 1e3)
                    batch.append(tm["batch_size"])
                wall = time.perf_counter() - t_start
            q = pcts(lat)
            lines.append({"offered_qps": lam, "queries": n, "achieved_qps": n / wall,
                          "p50_ms": q["p50"], "p90_ms": q["p90"], "p99_ms": q["p99"],
                          "rows_per_s": rows * n / wall,
                          "compressed_gbs": sum(alg[i] for i in pick) / wall / 1e9,
                          "mean_batch": float(np.mean(batch)), "mismatches_vs_alone": mismatch})
        return {"workload": w["name"], "fact_rows": rows, "fact_placement": placement,
                "query_variants": len(qs), "load_s": load_s, "rates": lines}
    finally:
        eng.close()


def run_serve(args, dpf, torch, np, local):
    """The serving sweep as its own run (``--serve``)."""
    rates = [float(x) for x in args.serve_rates.split(",")]
    r = serve_sweep(dpf, np, local, args.rows or (1 << 28), args.serve_placement, rates, args.serve_seconds,
                    args.serve_queries)
    out = {"metric": METRIC, "mode": "serve", "unit": "ms", "n_gpus": 1, "higher_is_better": False,
           "dtype": "int64", "data": "synthetic (seeded star schema; Poisson arrivals)",
           "config": {k: r[k] for k in ("workload", "fact_rows", "fact_placement", "query_variants", "load_s")},
           "rates": r["rates"]}
    print(json.dumps(out), flush=True)


def _fact_prefix(w, rows):
    """The workload with its fact table cut to the first ``rows`` rows."""
    import copy
    f = w["fact"]
    t = dict(w["tables"][f])
    cols = {}
    for name, c in t["cols"].items():
        if c["codec"] in ("str", "fsst"):
            offs = c["offsets"][: rows + 1]
            cols[name] = {"codec": "str", "bytes": c["bytes"][: int(offs[-1])], "offsets": offs}
        else:
            cols[name] = {"codec": c["codec"], "values": c["values"][:rows]}
    t["cols"], t["rows"] = cols, rows
    s = copy.copy(w)
    s["tables"] = dict(w["tables"])
    s["tables"][f] = t
    return s


def run_reference(args):
    """The CPU oracle as the reference arm, on every CPU of the process: each
    step decodes and evaluates a bounded prefix sample of the same workload
    (its pages encoded once beforehand by the oracle's own encoder, untimed),
    the sample sized from a short calibration so that the whole --warmup +
    --steps run takes about --ref-budget-s seconds."""
    import oracle
    w = _workload(args.workload, args.rows)
    n_total = w["tables"][w["fact"]]["rows"]
    cores, model = host_cpu()
    cal = _fact_prefix(w, min(n_total, 1 << 18))
    enc = oracle.encode_tables(cal)
    t0 = time.perf_counter()
    oracle.run_query(cal, encoded=enc, threads=cores)
    rate = cal["tables"][cal["fact"]]["rows"] / max(time.perf_counter() - t0, 1e-6)
    per_step_s = args.ref_budget_s / max(1, args.steps + args.warmup)
    rows = int(min(n_total, max(1 << 16, rate * per_step_s)))
    s = _fact_prefix(w, rows)
    enc = oracle.encode_tables(s)
    for _ in range(args.warmup):
        oracle.run_query(s, encoded=enc, threads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.run_query(s, encoded=enc, threads=cores)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = rows * len(times) / total
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic (seeded; stands in for SSB/TPC-H-style star schemas)",
        "config": {"workload": w["name"], "fact_rows": n_total, "sample_rows": rows},
        "cpu_baseline": {"value": value, "unit": "rows/s", "cores": cores, "kind": "oracle", "cpu_model": model,
                         "sample": f"first {rows} of {n_total} fact rows per step, decode + evaluate on {cores} "
                                   "threads (pages encoded beforehand, untimed)"},
        "e2e": {"value": value, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="dpf", choices=["dpf", "reference"])
    ap.add_argument("--workload", default="star",
                    choices=["star", "star_unsorted", "star_year", "star_year_unsorted", "star_bigint", "scan",
                             "strings", "strings_all", "groups_hot",
                             "strings_text", "strings_fsst", "chain", "chain_sparse", "batched"])
    ap.add_argument("--batch-queries", type=int, default=64)
    ap.add_argument("--batch-max-rows", type=int, default=None,
                    help="cap every batched query's fact rows (a smaller batch for profiling)")
    ap.add_argument("--serve", action="store_true", help="Poisson serving run instead of the step benchmark")
    ap.add_argument("--serve-rates", default="10,100,500,1000,2000")
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--serve-queries", type=int, default=2000)
    ap.add_argument("--serve-placement", default="device", choices=["device", "host"])
    ap.add_argument("--rows", type=int, default=0)
    ap.add_argument("--chunk-rows", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--ht", default="auto", choices=["auto", "smem", "global"])
    ap.add_argument("--ctas", type=int, default=0, help="CTAs per SM (4 = the 4-CTA kernel build)")
    ap.add_argument("--stage", default="default", choices=["default", "on", "off"],
                    help="stage the first step's mini blocks in shared memory (cp.async ring)")
    ap.add_argument("--group-agg", default="default", choices=["default", "warp", "atomic"],
                    help="grouped aggregates: warp-aggregated or one atomic per row")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-unfused", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the strings / batch / serving measurements that follow the headline")
    ap.add_argument("--ref-budget-s", type=float, default=120.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return

    import numpy as np
    import torch

    import paper_2605_10511_gb300 as dpf

    torch.cuda.set_device(local)
    if args.serve:
        if rank == 0:
            run_serve(args, dpf, torch, np, local)
        return
    if args.workload == "batched":
        if rank == 0:
            run_batched(args, dpf, torch, np, local)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    w = _workload(args.workload, args.rows)
    fact_rows = w["tables"][w["fact"]]["rows"]
    eng = dpf.Engine(device=local)
    eng.load_workload(w)
    stream = torch.cuda.Stream()
    chain = time_chain_builds(eng, w, stream, torch)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        plan = eng.plan(w, stream)
    torch.cuda.synchronize()
    build_ms = 1e3 * (time.perf_counter() - t0)
    autotuned = None
    if not _explicit_tuning(args):
        # the library's autotuner picks the launch configuration (cached
        # for this plan's signature; untimed)
        best, best_ms = eng.ctx.autotune([plan], stream, reps=3)
        autotuned = {"best": best, "best_ms": best_ms}
    tuning = dpf.Tuning(args.chunk_rows, args.threads, dpf.HT_PLACE[args.ht], args.ctas, dpf.STAGING[args.stage],
                        dpf.GROUP_AGG[args.group_agg])
    prep = eng.ctx.prepare([plan], tuning)
    eng.ctx.capture_graph(prep, stream)
    for _ in range(args.warmup):
        eng.ctx.launch_graph(prep, stream)
    records = eng.ctx.read_result(prep, 0)
    alg_bytes, _ = eng.fact_bytes(w)

    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        starts[i].record(stream)
        eng.ctx.launch_graph(prep, stream)
        ends[i].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    per = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = starts[0].elapsed_time(ends[-1])
    ms_step = total_ms / args.steps
    if world > 1:
        t = torch.tensor([ms_step], device=f"cuda:{local}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    check = eng.ctx.read_result(prep, 0)
    assert np.array_equal(check, records), "result changed across replays"
    # cold launches: 2 x L2 of device memory rewritten before each replay
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=f"cuda:{local}")
    cold = time_graph(eng.ctx, prep, stream, torch, max(10, min(args.steps, 30)), 1, flush=flush)
    del flush

    unfused = time_unfused(eng, plan, stream, records, reps=max(3, min(args.steps, 10)),
                           fused_ms=ms_step) if not args.no_unfused else None

    peak, peak_kind = _peaks()
    avg_launch_ms = statistics.mean(per)
    traffic, traffic_src = stored_traffic(args.workload, fact_rows)
    achieved = alg_bytes / (avg_launch_ms * 1e-3) / 1e9
    value = world * fact_rows / (ms_step * 1e-3)
    warm = pcts(per)
    out = {
        "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64",
        "data": "synthetic (seeded; stands in for SSB/TPC-H-style star schemas)",
        "config": {"workload": w["name"], "fact_rows": fact_rows, "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2 (compressed fact columns > 129 MB)"
                   if alg_bytes > 129e6 else "inputs smaller than L2",
                   "tuning": eng.ctx.prep_tuning(prep)},
        "compressed_gbs": achieved, "compressed_bytes": alg_bytes,
        "latency_ms": {"p50": warm["p50"], "p90": warm["p90"], "p99": warm["p99"], "mean": warm["mean"],
                       "how": "warm: back-to-back graph replays (the timed steps)",
                       "cold": dict(pcts(cold), how=f"{2 * L2_BYTES >> 20} MiB of device memory rewritten "
                                                    "on the stream before each replay (L2 flushed)")},
        "build_ms": build_ms,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_src,
                     "peak_kind": f"{peak_kind} copy bandwidth (burst)",
                     "frac_of_spec": achieved / SPEC_HBM_GBS, "spec_peak": SPEC_HBM_GBS,
                     "frac_cold": alg_bytes / (pcts(cold)["mean"] * 1e-3) / 1e9 / peak},
        "unfused": unfused,
        "autotune": autotuned,
        "gpu_launches": args.steps,
        "clocks": clocks,
        "wall_s": wall,
    }

    tuned = eng.ctx.prep_tuning(prep)
    eng.ctx.release(prep)
    if chain:
        link_ms = sum(x["ms"] for x in chain)
        rows_all = fact_rows + sum(x["rows"] for x in chain)
        out["chain"] = {"links": chain, "fused_ms": ms_step, "pipeline_ms": link_ms + ms_step,
                        "pipeline_rows_per_s": rows_all / ((link_ms + ms_step) * 1e-3)}
        for mode in ("exact", "async"):
            p = time_chain_pipeline(eng, w, stream, torch, np, records, asynchronous=mode == "async")
            p["rows_per_s"] = rows_all / (p["wall_ms"] * 1e-3)
            out["chain"][f"pipeline_{mode}"] = p
        p = time_chain_graph(eng, w, stream, torch, np, records, tuned)
        p["rows_per_s"] = rows_all / (p["wall_ms"] * 1e-3)
        out["chain"]["pipeline_graph"] = p
    links = None
    try:
        links = {"host_read_gbs": eng.ctx.read_rate("host", 2 << 30, 5, stream),
                 "device_read_gbs": eng.ctx.read_rate("device", 4 << 30, 5, stream),
                 "how": "dpf_read_rate: 16-byte read-only loads by every SM over 2 GiB of mapped pinned host "
                        "memory / 4 GiB of device memory, mean of 5 passes"}
        out["link_peaks"] = links
    except dpf.DpfError as e:
        out["link_peaks"] = {"unavailable": str(e)}
    eng.close()
    if not args.no_e2e:
        out["e2e"] = e2e_host_resident(dpf, w, args, local, tuning)
        if links and out["e2e"].get("value"):
            e = out["e2e"]
            step_s = fact_rows / e["value"]
            rate = e["h2d_bytes_per_step"] / step_s / 1e9
            e["page_bytes_gbs"] = rate
            e["page_bytes_frac_of_host_link"] = rate / links["host_read_gbs"]
            link, src = stored_link_bytes(args.workload, fact_rows)
            if link is None:
                t, tsrc = stored_traffic(args.workload, fact_rows)
                if t is not None:
                    link, src = t, ("estimate: the DRAM bytes of the HBM-resident kernel's capture of this query "
                                    f"({tsrc}); the host-resident kernel reads the same sectors over the link")
            if link is not None:
                # the kernel reads only the sectors holding a survivor's field of
                # the later steps' columns: the bytes that crossed the link
                e["link_bytes_per_step"] = link
                e["link_gbs"] = link / step_s / 1e9
                e["frac_of_host_link"] = e["link_gbs"] / links["host_read_gbs"]
                e["link_bytes_source"] = src
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baselines(w)
    if rank == 0 and world == 1 and not args.no_extras and args.workload == "star":
        out["extra"] = run_extras(args, dpf, torch, np, local)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _timed_workload(dpf, torch, np, local, w, steps, unfused_reps=3):
    """One query of workload w, autotuned, replayed from a CUDA graph: ms per
    launch (events on the launching stream), the fraction of the measured
    copy peak on its compressed bytes, and the unfused chain beside it."""
    peak, _ = _peaks()
    eng = dpf.Engine(device=local)
    try:
        eng.load_workload(w)
        stream = torch.cuda.Stream()
        plan = eng.plan(w, stream)
        best, _ = eng.ctx.autotune([plan], stream, reps=2)
        prep = eng.ctx.prepare([plan])
        eng.ctx.capture_graph(prep, stream)
        per = time_graph(eng.ctx, prep, stream, torch, steps, 3)
        rec = eng.ctx.read_result(prep, 0)
        tuned = eng.ctx.prep_tuning(prep)
        eng.ctx.release(prep)
        alg, rows = eng.fact_bytes(w)
        ms = statistics.mean(per)
        out = {"workload": w["name"], "ms": ms, "p50_ms": pcts(per)["p50"], "p90_ms": pcts(per)["p90"],
               "rows_per_s": rows / (ms * 1e-3), "compressed_gbs": alg / (ms * 1e-3) / 1e9,
               "frac": alg / (ms * 1e-3) / 1e9 / peak, "tuning": tuned}
        if unfused_reps:
            u = time_unfused(eng, plan, stream, rec, reps=unfused_reps, fused_ms=ms)
            out["unfused_ms"] = u.get("ms_per_query")
            out["fused_speedup"] = u.get("fused_speedup")
        return out
    finally:
        eng.close()


def run_extras(args, dpf, torch, np, local):
    """The other configurations, measured after the headline so they cannot
    disturb it: strings 2^25 (prefix filter; and every row passing, the
    warp-aggregated group-by under Zipf keys), the 64-query batch in one
    launch, and a short serving sweep over a 2^28-row star schema."""
    import synth
    ex = {}
    for name in ("strings", "strings_all"):
        try:
            ex[name] = _timed_workload(dpf, torch, np, local, _workload(name, 0), steps=20)
        except Exception as e:  # noqa: BLE001
            ex[name] = {"error": repr(e)}
    try:
        ws = synth.batched_workloads(n_queries=64, seed=4)
        eng = dpf.Engine(device=local)
        try:
            for w in ws:
                eng.load_workload(w)
            stream = torch.cuda.Stream()
            plans = [eng.plan(w, stream) for w in ws]
            eng.ctx.autotune(plans, stream, reps=1)
            prep = eng.ctx.prepare(plans)
            eng.ctx.capture_graph(prep, stream)
            per = time_graph(eng.ctx, prep, stream, torch, 5, 3)
            alg = sum(eng.fact_bytes(w)[0] for w in ws)
            rows = sum(w["tables"][w["fact"]]["rows"] for w in ws)
            ms = statistics.mean(per)
            peak, _ = _peaks()
            ex["batched_64"] = {"ms": ms, "rows": rows, "rows_per_s": rows / (ms * 1e-3),
                                "compressed_gbs": alg / (ms * 1e-3) / 1e9, "frac": alg / (ms * 1e-3) / 1e9 / peak,
                                "tuning": eng.ctx.prep_tuning(prep), "queries": len(ws)}
            eng.ctx.release(prep)
        finally:
            eng.close()
        del ws
    except Exception as e:  # noqa: BLE001
        ex["batched_64"] = {"error": repr(e)}
    try:
        ex["serving"] = serve_sweep(dpf, np, local, rows=1 << 28, placement="device", rates=(10.0, 500.0, 1000.0),
                                    seconds=1.5, max_queries=1500)
    except Exception as e:  # noqa: BLE001
        ex["serving"] = {"error": repr(e)}
    return ex


def time_chain_builds(eng, w, stream, torch, reps=5):
    """For a query whose joins form a chain: the wall time (median of
    ``reps``, host synchronisation included) of building each table, inner
    tables first: Kernel #1 (scan + build) for a table that probes nothing,
    Kernel #2 (scan + probe + build) for one that probes the tables built
    before it.  The last build of each link stays cached for the plan.
    Returns None when no join has joins of its own."""
    if not any(j.get("joins") for j in w["query"]["joins"]):
        return None
    links = []

    def walk(j):
        for s in j.get("joins", []):
            walk(s)
        sig = (w["name"], repr(j))
        times = []
        for _ in range(reps):
            old = eng.hts.pop(sig, None)
            if old is not None:
                eng.ctx.drop_hash(old)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ht = eng.build_join(w, j, stream)
            torch.cuda.synchronize()
            times.append(1e3 * (time.perf_counter() - t0))
        links.append({"table": j["dim"], "rows": w["tables"][j["dim"]]["rows"],
                      "kernel": "scan+probe+build" if j.get("joins") else "scan+build",
                      "entries": eng.ctx.hash_info(ht)["entries"], "ms": statistics.median(times)})

    for j in w["query"]["joins"]:
        walk(j)
    return links


def time_chain_pipeline(eng, w, stream, torch, np, want, asynchronous, reps=9):
    """A whole chain query from its tables to its records, as a user runs it
    once per query: the chain's tables are dropped, then built (with
    ``asynchronous``, enqueue-only builds sized from load-time bounds; else
    the exactly sized builds, which read each kept count back), the fused
    plan over the last table is prepared and launched on the same stream,
    its records are read and (async) every build's status is checked.
    ``wall_ms``: median host time of ``reps`` such queries; ``gpu_ms``:
    CUDA events from before the first build to after the fused launch.  An
    untimed first query autotunes the plan (the tuning is cached for its
    signature) and every query's records must equal ``want``."""
    def drop():
        for sig in [k for k in eng.hts if k[0] == w["name"]]:
            eng.ctx.drop_hash(eng.hts.pop(sig))

    walls, gpus = [], []
    for r in range(reps + 1):
        drop()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        plan = eng.plan(w, stream, asynchronous=asynchronous)
        if r == 0:
            eng.ctx.autotune([plan], stream, reps=2)
        prep = eng.ctx.prepare([plan])
        try:
            eng.ctx.launch(prep, stream)
            e1.record(stream)
            got = eng.ctx.read_result(prep, 0)
        finally:
            eng.ctx.release(prep)
        if asynchronous:
            eng.wait_joins(w)
        t1 = time.perf_counter()
        assert np.array_equal(got, want), "chain pipeline records differ"
        if r:
            walls.append(1e3 * (t1 - t0))
            gpus.append(e0.elapsed_time(e1))
    tables = []

    def walk(j):
        for s in j.get("joins", []):
            walk(s)
        tables.append(dict(eng.ctx.hash_info(eng.hts[(w["name"], repr(j))]), table=j["dim"]))
    for j in w["query"]["joins"]:
        walk(j)
    return {"wall_ms": statistics.median(walls), "gpu_ms": statistics.median(gpus), "reps": reps,
            "builds": "enqueue-only, sized from load-time bounds" if asynchronous else "exact (kept count read back)",
            "tables": tables}


def time_chain_graph(eng, w, stream, torch, np, want, tuning, reps=20):
    """The whole chain query as one prepared chain replayed from one CUDA
    graph: every replay rebuilds CUSTOMER's and ORDERS' tables (Kernels #1
    and #2, enqueue-only sizing) and runs the fused plan over LINEITEM
    (Kernel #3), then the records are read and each build's status checked.
    ``wall_ms``: median host time from the replay to the checked records;
    ``gpu_ms``: CUDA events around the replay.  The plan runs at ``tuning``
    (the headline plan's autotuned configuration)."""
    prep = eng.prepare_chain(w, dpf_tuning(tuning))
    try:
        eng.ctx.launch(prep, stream)
        assert np.array_equal(eng.ctx.read_result(prep, 0), want), "prepared chain records differ"
        eng.wait_joins(w, deferred=True)
        eng.ctx.capture_graph(prep, stream)
        walls, gpus = [], []
        for r in range(reps + 2):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            e0.record(stream)
            eng.ctx.launch_graph(prep, stream)
            e1.record(stream)
            got = eng.ctx.read_result(prep, 0)
            eng.wait_joins(w, deferred=True)
            t1 = time.perf_counter()
            assert np.array_equal(got, want), "prepared chain records differ"
            if r >= 2:
                walls.append(1e3 * (t1 - t0))
                gpus.append(e0.elapsed_time(e1))
        tables = [dict(eng.ctx.hash_info(h)) for h in eng.chain_tables(w, deferred=True)]
    finally:
        eng.ctx.release(prep)
    return {"wall_ms": statistics.median(walls), "gpu_ms": statistics.median(gpus), "reps": reps,
            "builds": "deferred tables rebuilt by every replay of one CUDA graph", "tables": tables}


def dpf_tuning(t):
    """A Tuning structure from the dict dpf_prep_tuning returns."""
    import paper_2605_10511_gb300 as dpf
    return dpf.Tuning(t["chunk_rows"], t["threads"], t["ht_placement"], t["ctas_per_sm"], t["staging"],
                      t["group_agg"])


def time_unfused(eng, plan, stream, fused_records, reps, fused_ms):
    """The same plan through the unfused per-operator chain (one kernel per
    operator, intermediates in HBM): time per query, kernel launches and
    intermediate bytes, checked against the fused result."""
    import numpy as np
    import torch
    import paper_2605_10511_gb300 as dpf
    try:
        prep = eng.ctx.prepare_unfused(plan)
    except dpf.DpfError as e:  # the chain evaluates PREFIX on STR columns only
        return {"unsupported": str(e)}
    try:
        for _ in range(2):
            eng.ctx.launch(prep, stream)
        got = eng.ctx.read_result(prep, 0)
        assert np.array_equal(got, fused_records), "unfused chain disagrees with the fused kernel"
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        s.record(stream)
        for _ in range(reps):
            eng.ctx.launch(prep, stream)
        e.record(stream)
        torch.cuda.synchronize()
        ms = s.elapsed_time(e) / reps
        st = eng.ctx.prep_stats(prep)
        return {"ms_per_query": ms, "launches_per_query": st["launches"],
                "intermediate_bytes": st["intermediate_bytes"], "fused_speedup": ms / fused_ms}
    finally:
        eng.ctx.release(prep)


def e2e_host_resident(dpf, w, args, device, tuning):
    """The same query through the public API with the fact pages in pinned
    host memory: every step the kernel reads the compressed pages over the
    host link and the records come back to the host."""
    import copy

    import torch
    w2 = copy.copy(w)
    w2["name"] = w["name"] + "_host"
    if tuning is not None and tuning.threads > 256:  # the wide CTAs take device-resident pages only
        tuning = dpf.Tuning(tuning.chunk_rows, 0, tuning.ht_placement, 0, tuning.staging, tuning.group_agg)
    eng = dpf.Engine(device=device)
    try:
        eng.load_workload(w2, fact_placement="host")
        stream = torch.cuda.Stream()
        plan = eng.plan(w2, stream)
        prep = eng.ctx.prepare([plan], tuning)
        for _ in range(args.warmup):
            eng.ctx.launch(prep, stream)
            eng.ctx.read_result(prep, 0)
        steps = max(3, min(args.steps, 20))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nrec = 0
        for _ in range(steps):
            eng.ctx.launch(prep, stream)
            nrec = len(eng.ctx.read_result(prep, 0))
        dt = time.perf_counter() - t0
        bytes_in, rows = eng.fact_bytes(w2)
        eng.ctx.release(prep)
        return {"value": rows * steps / dt, "unit": "rows/s", "h2d_bytes_per_step": int(bytes_in),
                "d2h_bytes_per_step": int(nrec * 48 + 12), "how": "fact pages in pinned host memory "
                "read in-kernel; records copied to host each step"}
    finally:
        eng.close()


if __name__ == "__main__":
    main()
