"""Sharded runs on CPU ranks (gloo, world size 2): each rank evaluates its
contiguous range of fact pages, the ranks exchange their int64 group
records, and the merge equals the whole table's result (star, strings,
random small workloads, a join chain, a BIGINT measure).  The oracle stands
in for each rank's fused kernel; what is tested is the host logic of
sharding and merging (paper_2605_10511_gb300.replicas)."""

import os
import socket

import numpy as np
import pytest

import oracle
import synth
from paper_2605_10511_gb300 import RECORD_DTYPE
from paper_2605_10511_gb300.replicas import merge_records, shard_rows, slice_workload


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workloads():
    ws = [synth.tiny_random_workload(s, rows=9000, page_rows=1024) for s in (3, 8, 21)]
    ws.append(synth.star_join(rows=70000, seed=9, page_rows=4096))
    ws.append(synth.strings(rows=50000, seed=9, page_rows=2048))
    # a join chain: each rank builds the whole inner tables and scans its
    # part of LINEITEM; a BIGINT measure
    ws.append(synth.chain_join(rows=60000, seed=9, page_rows=2048))
    ws.append(synth.star_join(rows=40000, seed=10, page_rows=2048, bigint_measure=True))
    return ws


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        for i, w in enumerate(_workloads()):
            t = w["tables"][w["fact"]]
            lo, hi = shard_rows(t["rows"], t["page_rows"], rank, world)
            part = oracle.run_query(slice_workload(w, lo, hi), from_encoded=True)
            parts = [None] * world
            dist.all_gather_object(parts, part.tobytes())
            merged = merge_records([np.frombuffer(b, RECORD_DTYPE) for b in parts], bool(w["query"]["group"]))
            if rank == 0:
                out[i] = merged.tobytes()
    finally:
        dist.destroy_process_group()


def test_shard_rows_cover_the_table_with_whole_pages():
    for nrows, pr in ((1, 128), (1000, 128), (65536 * 3 + 5, 65536), (4096, 4096)):
        for world in (1, 2, 3, 8):
            spans = [shard_rows(nrows, pr, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == nrows
            for (a, b), (c, d) in zip(spans, spans[1:]):
                assert b == c and a <= b
            assert all(a % pr == 0 for a, _ in spans)


def test_merge_of_two_gloo_ranks_equals_whole_table():
    import torch.multiprocessing as mp
    oracle.build()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    for i, w in enumerate(_workloads()):
        want = oracle.run_query(w, from_encoded=False)
        got = np.frombuffer(out[i], RECORD_DTYPE)
        assert got.shape == want.shape, w["name"]
        for f in ("key", "count", "val"):
            assert np.array_equal(got[f], want[f]), (w["name"], f)


def test_merge_keeps_one_record_for_empty_ungrouped_queries():
    empty = np.zeros(1, RECORD_DTYPE)
    m = merge_records([empty, empty], grouped=False)
    assert m.shape == (1,) and m["count"][0] == 0
    a = np.zeros(2, RECORD_DTYPE)
    a["key"] = [[1, 0], [3, 0]]
    a["count"] = [2, 5]
    b = np.zeros(1, RECORD_DTYPE)
    b["key"] = [[2, 0]]
    b["count"] = [7]
    m = merge_records([a, b], grouped=True)
    assert m["key"][:, 0].tolist() == [1, 2, 3] and m["count"].tolist() == [2, 7, 5]
