"""GPU parity of plans with predicates every row passes, and the context's
default launch configuration.

The planner compiles an empty PREFIX or CONTAINS pattern, LIKE '%', and a
range over a column's whole int32 or int64 domain to no step at all (the
column is checked, not read); a grouped scan with no other filter then
leads with its group key.  Records must equal the oracle's and those of the
same query without the predicate, a dropped predicate on a column of
another table must still be refused, and a plan left with no step at all
must count every row.
"""

import copy

import numpy as np
import pytest

import oracle
import paper_2605_10511_gb300 as dpf
import synth

pytestmark = pytest.mark.gpu

I32_MIN, I32_MAX = -(1 << 31), (1 << 31) - 1


def assert_same(got, want, what=""):
    assert got.shape == want.shape, (what, got, want)
    for f in ("key", "count", "val"):
        assert np.array_equal(got[f], want[f]), (what, f)


@pytest.fixture(scope="module")
def eng():
    e = dpf.Engine(device=0)
    yield e
    e.close()


@pytest.fixture(scope="module")
def strings_w():
    return synth.strings(rows=(1 << 20) + 99, page_rows=65536, prefix=b"", seed=21)


ALWAYS = {
    "empty_prefix": {"col": "s", "op": "prefix", "args": [b""]},
    "like_percent": {"col": "s", "op": "like", "args": [b"%"]},
    "like_percents": {"col": "s", "op": "like", "args": [b"%%%"]},
    "empty_contains": {"col": "s", "op": "contains", "args": [b""]},
    "full_int32_range": {"col": "m", "op": "between", "args": [I32_MIN, I32_MAX]},
    "ge_int32_min": {"col": "m", "op": "ge", "args": [I32_MIN]},
}


@pytest.mark.parametrize("case", sorted(ALWAYS))
def test_always_true_predicates_match_the_plan_without_them(eng, strings_w, case):
    w = copy.deepcopy(strings_w)
    w["query"]["preds"] = [ALWAYS[case]]
    bare = copy.deepcopy(strings_w)
    bare["query"]["preds"] = []
    want = oracle.run_query(w, from_encoded=False, threads=0)
    assert_same(want, oracle.run_query(bare, from_encoded=False, threads=0), case)
    assert_same(eng.run(w), want, case)
    assert_same(eng.run(bare), want, (case, "bare"))


def test_with_a_real_filter_beside_it(eng, strings_w):
    w = copy.deepcopy(strings_w)
    w["query"]["preds"] = [ALWAYS["like_percent"], {"col": "m", "op": "lt", "args": [250000]},
                           ALWAYS["full_int32_range"]]
    assert_same(eng.run(w), oracle.run_query(w, from_encoded=False, threads=0))


def test_bigint_domain_predicates():
    w = synth.bigint_filter_star((1 << 20) + 7, 5, 65536, joins=False,
                                 preds=[{"col": "m1", "op": "ge", "args": [-(1 << 63)]},
                                        {"col": "m1", "op": "le", "args": [(1 << 63) - 1]}])
    e = dpf.Engine(device=0)
    try:
        got = e.run(w)
        assert_same(got, oracle.run_query(w, from_encoded=False, threads=0))
        assert int(got["count"][0]) == w["tables"]["fact"]["rows"]
    finally:
        e.close()


def test_no_step_at_all_counts_every_row(eng, strings_w):
    w = copy.deepcopy(strings_w)
    w["query"]["preds"] = [ALWAYS["empty_prefix"]]
    w["query"]["group"] = []
    w["query"]["aggs"] = [{"op": "count"}]
    got = eng.run(w)
    assert_same(got, oracle.run_query(w, from_encoded=False, threads=0))
    assert int(got["count"][0]) == w["tables"]["fact"]["rows"]


def test_a_dropped_predicate_is_still_checked(eng, strings_w):
    """An always-true predicate on a column of another table is refused."""
    other = synth.scan_filter_aggregate(rows=5000, page_rows=4096, seed=22)
    eng.load_workload(strings_w)
    eng.load_workload(other)
    h = eng.plan(strings_w)
    preds = (dpf.Pred * 1)(dpf.make_pred(eng.col(other, "fact", "a"), "between", [I32_MIN, I32_MAX]))
    h.plan.n_preds = 1
    h.plan.preds = dpf.C.cast(preds, dpf.C.POINTER(dpf.Pred))
    h._keep = (h._keep, preds)
    with pytest.raises(dpf.DpfError) as e:
        eng.ctx.prepare([h])
    assert e.value.status == -1


def test_context_default_tuning(strings_w):
    """dpf_set_tuning: a prepare without a tuning takes the context's
    defaults (the fields it leaves open), an explicit tuning overrides them,
    a reset restores the library's; records stay the oracle's."""
    w = copy.deepcopy(strings_w)
    w["query"]["preds"] = [{"col": "s", "op": "prefix", "args": [b"q"]}]
    want = oracle.run_query(w, from_encoded=False, threads=0)
    e = dpf.Engine(device=0)
    try:
        e.load_workload(w)
        h = e.plan(w)

        def run(tuning=None):
            prep = e.ctx.prepare([h], tuning)
            try:
                e.ctx.launch(prep)
                assert_same(e.ctx.read_result(prep, 0), want)
                return e.ctx.prep_tuning(prep)
            finally:
                e.ctx.release(prep)
        e.ctx.set_tuning({"chunk_rows": 8192, "threads": 128, "ht_placement": "global"})
        t = run()
        assert (t["chunk_rows"], t["threads"], t["ht_placement"]) == (8192, 128, 2)
        t = run(dpf.Tuning(2048, 256, 0, 0, 0, 0))
        assert (t["chunk_rows"], t["threads"], t["ht_placement"]) == (2048, 256, 2)
        with pytest.raises(dpf.DpfError):
            e.ctx.set_tuning('{"threads": 300}')
        t = run()  # a refused object leaves the defaults as they were
        assert (t["chunk_rows"], t["threads"]) == (8192, 128)
        e.ctx.set_tuning(None)
        t = run()
        assert (t["chunk_rows"], t["threads"], t["ht_placement"]) == (4096, 256, 0)
    finally:
        e.close()
