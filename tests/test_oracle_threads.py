"""The oracle's threaded walk equals its one-thread definition (CPU only).

``orc_query_threads`` cuts the fact rows into page ranges, evaluates them
on several host threads into separate group maps and adds the maps
together.  Integer addition modulo 2^64 is associative, so its records must
be identical to ``orc_query``'s, the plain row-at-a-time walk, for every
thread count, including more threads than ranges, ranges that end in a
ragged page, ungrouped queries with no surviving row and sums that wrap.
"""

import numpy as np
import pytest

import npeval
import oracle
import synth


def _same(a, b, what):
    assert a.shape == b.shape, (what, a, b)
    for f in ("key", "count", "val"):
        assert np.array_equal(a[f], b[f]), (what, f)


@pytest.mark.parametrize("threads", [2, 3, 8, 64])
def test_threads_equal_one_thread_on_random_workloads(oracle_lib, threads):
    for seed in range(40):
        w = synth.tiny_random_workload(seed)
        one = oracle.run_query(w, from_encoded=False)
        _same(oracle.run_query(w, from_encoded=False, threads=threads), one, ("random", seed))
        _same(one, npeval.evaluate(w), ("numpy", seed))


def test_threads_equal_one_thread_on_chains(oracle_lib):
    for seed in range(24):
        w = synth.tiny_chain_workload(seed)
        _same(oracle.run_query(w, from_encoded=False, threads=5),
              oracle.run_query(w, from_encoded=False), ("chain", seed))


@pytest.mark.parametrize("shape", ["scan", "star", "strings", "star_unsorted"])
def test_threads_equal_one_thread_on_bench_shapes(oracle_lib, shape):
    """Tables of several pages with a ragged last page, as the full-size
    tests evaluate them (every CPU of the process)."""
    w = {"scan": lambda: synth.scan_filter_aggregate(rows=300_001, page_rows=4096),
         "star": lambda: synth.star_join(rows=400_003, page_rows=8192),
         "strings": lambda: synth.strings(rows=200_017, page_rows=16384),
         "star_unsorted": lambda: synth.star_join(rows=250_000, page_rows=2048, clustered=False)}[shape]()
    one = oracle.run_query(w, from_encoded=False)
    _same(oracle.run_query(w, from_encoded=False, threads=0), one, shape)
    _same(oracle.run_query(w, from_encoded=False, threads=7), one, shape)


def test_threads_empty_result_and_wrapping_sums(oracle_lib):
    """An ungrouped query whose filter keeps nothing still yields one record
    of zeros; sums that pass 2^63 wrap identically on both walks."""
    n = 5000
    big = np.full(n, 2**62 + 12345, np.int64)
    w = {"name": "wrap", "fact": "f", "tables": {"f": {"rows": n, "page_rows": 256, "cols": {
        "a": {"codec": "for", "values": np.arange(n, dtype=np.int32)},
        "g": {"codec": "dict", "values": (np.arange(n) % 3).astype(np.int32)},
        "b": {"codec": "for64", "values": big}}}},
        "query": {"preds": [], "joins": [], "group": [{"col": "g"}],
                  "aggs": [{"op": "sum", "cols": ["b"]}, {"op": "sum_mul", "cols": ["b", "a"]}]}}
    one = oracle.run_query(w, from_encoded=False)
    _same(oracle.run_query(w, from_encoded=False, threads=4), one, "wrap")
    counts = np.bincount(np.arange(n) % 3)
    want = [int(np.uint64((2**62 + 12345) * int(c) % 2**64).astype(np.int64)) for c in counts]
    assert one["val"][:, 0].tolist() == want
    w["query"] = {"preds": [{"col": "a", "op": "lt", "args": [-1]}], "joins": [], "group": [],
                  "aggs": [{"op": "count"}]}
    r = oracle.run_query(w, from_encoded=False, threads=4)
    assert r.shape == (1,) and r["count"][0] == 0 and not r["val"].any()


def test_threaded_decode_equals_one_thread(oracle_lib):
    """Decoding integer columns page range by page range on several threads
    gives the one-thread decoder's rows, for every integer codec and ragged
    last pages; a query over pre-encoded pages agrees too."""
    w = synth.star_join(rows=300_007, page_rows=4096, bigint_measure=True)
    enc = oracle.encode_tables(w)
    for (t, c), e in enc.items():
        if e["codec"] in ("str", "fsst"):
            continue
        one = oracle.decode_column(e)
        for threads in (2, 7, 1000):
            assert np.array_equal(oracle.decode_column(e, threads=threads), one), (t, c, threads)
    one = oracle.run_query(w, from_encoded=False)
    _same(oracle.run_query(w, encoded=enc, threads=5), one, "encoded, threads")
    _same(oracle.run_query(w, encoded=enc), one, "encoded")
