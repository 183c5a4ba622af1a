"""Pins of the oracle's query evaluator (CPU only).

* brute force on small tables: an independent numpy evaluator (``npeval``)
  built on library routines (masks, searchsorted joins, np.unique grouping,
  np.add.at sums) must give exactly the same records;
* the oracle evaluated on its own encoded-then-decoded columns equals the
  oracle evaluated on the raw arrays (checks the encoder/decoder pair);
* invariants: group counts sum to the filtered-and-joined row count; group
  sums add up to the ungrouped sum; all-pass predicates over complete
  dimensions count every fact row; a filtered build equals an unfiltered
  build followed by the same filter; a clustered (sorted) fact table gives
  the same result as its unsorted copy;
* special cases reducing to library routines: an unfiltered ungrouped SUM is
  ``numpy.sum`` in int64; a single-key COUNT is ``numpy.bincount``.
"""

import copy

import numpy as np
import pytest

import npeval
import synth


def _records_equal(a, b):
    assert a.shape == b.shape, (a, b)
    assert np.array_equal(a["key"], b["key"]), (a["key"], b["key"])
    assert np.array_equal(a["count"], b["count"]), (a["count"], b["count"])
    assert np.array_equal(a["val"], b["val"]), (a["val"], b["val"])


@pytest.mark.parametrize("seed", range(40))
def test_oracle_matches_numpy_on_tiny_tables(oracle_lib, seed):
    w = synth.tiny_random_workload(seed)
    expect = npeval.evaluate(w)
    got_raw = oracle_lib.run_query(w, from_encoded=False)
    got_enc = oracle_lib.run_query(w, from_encoded=True)
    _records_equal(got_raw, expect)
    _records_equal(got_enc, expect)


def test_scan_filter_aggregate_small(oracle_lib):
    w = synth.scan_filter_aggregate(rows=50000, seed=1, page_rows=4096)
    got = oracle_lib.run_query(w)
    _records_equal(got, npeval.evaluate(w))
    c = w["tables"]["fact"]["cols"]
    a, b = c["a"]["values"], c["b"]["values"]
    m = (a < 25) & (b >= 1) & (b <= 3)
    assert int(got["count"][0]) == int(m.sum())
    assert int(got["val"][0, 0]) == int((c["c"]["values"][m].astype(np.int64)
                                        * c["d"]["values"][m].astype(np.int64)).sum())


def test_star_join_small_and_invariants(oracle_lib):
    w = synth.star_join(rows=200000, seed=2, page_rows=8192, clustered=False,
                        dim_rows=(2000, 30000, 20000))
    got = oracle_lib.run_query(w)
    _records_equal(got, npeval.evaluate(w))
    # clustered copy: same result
    wc = synth.star_join(rows=200000, seed=2, page_rows=8192, clustered=True,
                         dim_rows=(2000, 30000, 20000))
    _records_equal(oracle_lib.run_query(wc), got)
    # ungrouped variant: counts and sums add up
    wu = copy.deepcopy(w)
    wu["query"]["group"] = []
    u = oracle_lib.run_query(wu)
    assert u.shape == (1,)
    assert int(u["count"][0]) == int(got["count"].sum())
    assert int(u["val"][0, 0]) == int(got["val"][:, 0].sum())
    # unfiltered build + the same predicate on the fact side through a payload
    # cannot be expressed on the fact table, so check instead that dropping
    # every dimension predicate keeps every fact row (complete dimensions)
    wa = copy.deepcopy(w)
    for j in wa["query"]["joins"]:
        j["preds"] = []
    wa["query"]["group"] = []
    wa["query"]["aggs"] = [{"op": "count"}, {"op": "sum", "cols": ["m1"]}]
    a = oracle_lib.run_query(wa)
    fact = w["tables"]["fact"]["cols"]
    assert int(a["count"][0]) == w["tables"]["fact"]["rows"]
    assert int(a["val"][0, 1]) == int(fact["m1"]["values"].astype(np.int64).sum())


def test_strings_small(oracle_lib):
    w = synth.strings(rows=100000, seed=3, page_rows=4096)
    got = oracle_lib.run_query(w)
    _records_equal(got, npeval.evaluate(w))
    # grouped COUNT over all rows is np.bincount over the key codes
    wa = copy.deepcopy(w)
    wa["query"]["preds"] = []
    a = oracle_lib.run_query(wa)
    key = w["tables"]["fact"]["cols"]["key"]["values"]
    vals, counts = np.unique(key, return_counts=True)
    assert np.array_equal(a["key"][:, 0], vals)
    assert np.array_equal(a["count"], counts)
    assert int(got["count"].sum()) <= int(a["count"].sum())


def test_empty_prefix_selects_all_and_long_prefix_none(oracle_lib):
    w = synth.strings(rows=5000, seed=5, page_rows=1024)
    w["query"]["preds"] = [{"col": "s", "op": "prefix", "args": [b""]}]
    w["query"]["group"] = []
    assert int(oracle_lib.run_query(w)["count"][0]) == 5000
    w["query"]["preds"] = [{"col": "s", "op": "prefix", "args": [b"a" * 45]}]
    r = oracle_lib.run_query(w)
    assert r.shape == (1,) and int(r["count"][0]) == 0 and int(r["val"][0, 1]) == 0


def test_duplicate_build_keys_rejected(oracle_lib):
    w = synth.tiny_random_workload(3, rows=500, page_rows=128)
    w["query"]["joins"] = [{"fk": "fk", "dim": "dim", "key": "k", "preds": [], "payload": []}]
    w["query"]["group"] = []
    k = w["tables"]["dim"]["cols"]["k"]["values"]
    k[1] = k[0]
    with pytest.raises(oracle_lib.OracleError):
        oracle_lib.run_query(w, from_encoded=False)


def test_config1_statistical_sanity(oracle_lib):
    """Not parity: the 2^20-row scan selects about 2^20 * 24/50 * 3/50 rows."""
    w = synth.scan_filter_aggregate()
    r = oracle_lib.run_query(w)
    n = 1 << 20
    p = 24 / 50 * 3 / 50
    mean, sd = n * p, (n * p * (1 - p)) ** 0.5
    assert abs(int(r["count"][0]) - mean) < 5 * sd
    avg = int(r["val"][0, 0]) / int(r["count"][0])
    assert abs(avg - 5.5 * 52950) < 0.05 * 5.5 * 52950


@pytest.mark.parametrize("clustered", [True, False])
def test_star_join_with_date_filter(oracle_lib, clustered):
    """The one-year date filter: equal to the numpy evaluator, and the
    year key of every record is the filtered year."""
    w = synth.star_join(rows=60000, page_rows=4096, clustered=clustered, date_year=1995)
    got = oracle_lib.run_query(w, from_encoded=True)
    _records_equal(got, npeval.evaluate(w))
    assert got.shape[0] > 0 and np.all(got["key"][:, 1] == 1995)


def test_bigint_aggregates_wrap_modulo_2_64(oracle_lib):
    """Closed forms for FOR64 (BIGINT) operands: four copies of 2^62 sum to
    2^64 = 0 modulo 2^64; (2^32)^2 = 2^64 wraps to 0 as well; INT64_MIN - 1
    wraps to INT64_MAX; and a mixed 32/64-bit product keeps all 64 bits."""
    i64 = np.iinfo(np.int64)
    z = np.array([1 << 62] * 4 + [1 << 32, i64.min, 3 << 40], np.int64)
    x = np.array([1, 1, 1, 1, 1 << 30, 1, -7], np.int32)
    g = np.array([0, 0, 0, 0, 1, 2, 3], np.int32)
    w = {"name": "bigint_wrap", "fact": "f",
         "tables": {"f": {"rows": 7, "page_rows": 128,
                          "cols": {"z": {"codec": "for64", "values": z}, "x": {"codec": "for", "values": x},
                                   "g": {"codec": "dict", "values": g},
                                   "one": {"codec": "for", "values": np.ones(7, np.int32)}}}},
         "query": {"preds": [], "joins": [], "group": [{"col": "g"}],
                   "aggs": [{"op": "sum", "cols": ["z"]}, {"op": "sum_mul", "cols": ["z", "z"]},
                            {"op": "sum_sub", "cols": ["z", "one"]}, {"op": "sum_mul", "cols": ["z", "x"]}]}}
    for from_encoded in (False, True):
        r = oracle_lib.run_query(w, from_encoded=from_encoded)
        assert r["key"][:, 0].tolist() == [0, 1, 2, 3]
        assert r["count"].tolist() == [4, 1, 1, 1]
        # group 0: 4 * 2^62 = 2^64 -> 0; (2^62)^2 * 4 -> 0; 4 * (2^62 - 1) = 2^64 - 4 -> -4; 4 * 2^62 -> 0
        assert r["val"][0].tolist() == [0, 0, -4, 0]
        # group 1: 2^32; (2^32)^2 = 2^64 -> 0; 2^32 - 1; 2^32 * 2^30 = 2^62
        assert r["val"][1].tolist() == [1 << 32, 0, (1 << 32) - 1, 1 << 62]
        # group 2: INT64_MIN; INT64_MIN^2 = 2^126 -> 0; INT64_MIN - 1 -> INT64_MAX; INT64_MIN * 1
        assert r["val"][2].tolist() == [int(i64.min), 0, int(i64.max), int(i64.min)]
        # group 3: 3 * 2^40; 9 * 2^80 -> 0 mod 2^64; 3 * 2^40 - 1; -21 * 2^40
        assert r["val"][3].tolist() == [3 << 40, 0, (3 << 40) - 1, -21 * (1 << 40)]
