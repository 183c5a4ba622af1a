"""Parity at the full sizes of the benchmark configurations, in the launch
configuration bench.py times (default tuning, one persistent launch replayed
from a CUDA graph): scan-filter-aggregate 2^20 rows, star join 2^26 rows
(clustered, delta-coded dates; and with the fact pages in pinned host
memory), strings 2^25 rows, the 64-query batch (654 M fact rows in one
launch), and the serving mix through the continuous-batching server over a
2^28-row star schema in HBM and a 2^30-row one in pinned host memory (the
only tables whose page offsets pass 2^32 bytes).  Every record of every
query is compared with the oracle, which evaluates the whole table from the
generated arrays on every host CPU (its threaded walk, pinned equal to the
one-thread definition by the CPU tests)."""

import random
import threading
import time

import numpy as np
import pytest
import torch

import oracle
import paper_2605_10511_gb300 as dpf
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def assert_same(got, want, what=""):
    assert got.shape == want.shape, (what, got, want)
    for f in ("key", "count", "val"):
        assert np.array_equal(got[f], want[f]), (what, f)


def run_like_bench(eng, w, placement=None):
    eng.load_workload(w, fact_placement=placement)
    stream = torch.cuda.Stream()
    plan = eng.plan(w, stream)
    prep = eng.ctx.prepare([plan])
    try:
        eng.ctx.capture_graph(prep, stream)
        for _ in range(3):
            eng.ctx.launch_graph(prep, stream)
        return eng.ctx.read_result(prep, 0)
    finally:
        eng.ctx.release(prep)


@pytest.mark.parametrize("name", ["scan", "star", "strings"])
def test_full_size_matches_oracle(name):
    w = {"scan": lambda: synth.scan_filter_aggregate(rows=1 << 20),
         "star": lambda: synth.star_join(rows=1 << 26),
         "strings": lambda: synth.strings(rows=1 << 25)}[name]()
    want = oracle.run_query(w, from_encoded=False, threads=0)
    eng = dpf.Engine(device=0)
    try:
        assert_same(run_like_bench(eng, w), want, name)
        if name == "star":  # the end-to-end variant: pages in pinned host memory
            wh = dict(w, name=w["name"] + "_host")
            assert_same(run_like_bench(eng, wh, placement="host"), want, name + " host")
    finally:
        eng.close()


def test_full_size_batch_of_64():
    ws = synth.batched_workloads(n_queries=64, seed=4)
    eng = dpf.Engine(device=0)
    try:
        for w in ws:
            eng.load_workload(w)
        plans = [eng.plan(w) for w in ws]
        prep = eng.ctx.prepare(plans)
        stream = torch.cuda.Stream()
        eng.ctx.capture_graph(prep, stream)
        eng.ctx.launch_graph(prep, stream)
        batched = [eng.ctx.read_result(prep, i) for i in range(len(ws))]
        eng.ctx.release(prep)
        for i, w in enumerate(ws):
            assert_same(batched[i], oracle.run_query(w, from_encoded=False, threads=0), w["name"])
    finally:
        eng.close()


def _serve(eng, plans, order, rate_qps, seed):
    """Submits plans[order[k]] as a Poisson stream at ``rate_qps`` from two
    threads through the continuous-batching server; returns each ticket's
    records and the launch sizes seen."""
    rng = random.Random(seed)
    tickets = [None] * len(order)
    with dpf.Server(eng.ctx, max_batch=64, max_inflight=2) as srv:
        def submitter(part):
            for k in part:
                tickets[k] = srv.submit(plans[order[k]])
                time.sleep(rng.expovariate(rate_qps / 2))
        idx = list(range(len(order)))
        ts = [threading.Thread(target=submitter, args=(idx[j::2],)) for j in range(2)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        got, sizes = [], []
        for tk in tickets:
            r, times = srv.wait(tk, timeout_ms=600000)
            got.append(r)
            sizes.append(times["batch_size"])
        assert srv.stats()["failed"] == 0
    return got, sizes


@pytest.mark.parametrize("rows,placement", [(1 << 28, "device"), (1 << 30, "host")])
def test_full_size_serving_mix_matches_oracle(rows, placement):
    """The serving configuration: 16 query variants (12 star joins with
    re-drawn dimension predicates, 4 scan-filter-aggregates over the
    measures) over one resident star schema; 48 requests arrive as a
    Poisson stream and are batched by the server; every result equals the
    oracle's records for its query."""
    w = synth.star_join(rows=rows, clustered=placement == "device")
    qs = synth.serve_variants(w, 12, 4, seed=5)
    eng = dpf.Engine(device=0)
    try:
        eng.load_workload(w, fact_placement=placement)
        plans = [eng.plan(v) for v in qs]
        order = [k % len(qs) for k in range(3 * len(qs))]
        random.Random(rows).shuffle(order)
        got, sizes = _serve(eng, plans, order, rate_qps=400.0 if placement == "device" else 40.0, seed=rows)
        want = [oracle.run_query(v, from_encoded=False, threads=0) for v in qs]
        for k, q in enumerate(order):
            assert_same(got[k], want[q], (placement, k, q))
        assert sum(int(r["count"].sum()) for r in want) > 0
    finally:
        eng.close()
