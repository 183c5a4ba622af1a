"""GPU parity of predicates on BIGINT (FOR64) columns (Sec. 3.4.1, 4.1).

A predicate on a 64-bit GPU-FOR column compares the int64 value with int64
operands.  It runs over the survivors of the plan's 32-bit steps; when every
filter is 64-bit a pass-all first step leads.  Records must equal the
oracle's bit for bit: bounds below, across and above 2^32, every
comparison, empty and full selections, after the star's joins and as the
only filter, under the launch knobs, with host-resident pages, in a batch
next to 32-bit plans, in a dimension build (with and without a 32-bit
predicate beside it), at 2^25 fact rows; the unfused chain and IN lists
refuse them.
"""

import numpy as np
import pytest

import oracle
import paper_2605_10511_gb300 as dpf
import synth
from test_oracle_for64_preds import CASES, DIM_CASES, with_dim_bigint

pytestmark = pytest.mark.gpu

ROWS = (1 << 20) + 333  # 16 pages of 65,536 rows and a ragged one


def assert_same(got, want, what=""):
    assert got.shape == want.shape, (what, got, want)
    for f in ("key", "count", "val"):
        assert np.array_equal(got[f], want[f]), (what, f)


@pytest.fixture(scope="module")
def eng():
    e = dpf.Engine(device=0)
    yield e
    e.close()


def _w(case, joins, rows=ROWS, seed=7):
    return synth.bigint_filter_star(rows, seed, 65536, preds=CASES[case](), joins=joins)


@pytest.mark.parametrize("joins", [True, False])
@pytest.mark.parametrize("case", sorted(CASES))
def test_matches_oracle(eng, case, joins):
    # CASES take their equality operands from the 20,000-row table of seed 7;
    # this table shares its first rows' generator, so some may not occur: the
    # oracle decides either way
    w = _w(case, joins)
    assert_same(eng.run(w), oracle.run_query(w, from_encoded=False, threads=0), (case, joins))


@pytest.mark.parametrize("cfg", [dict(threads=1024), dict(threads=256, ctas_per_sm=4), dict(threads=128),
                                 dict(ht_placement=2), dict(staging=1)])
@pytest.mark.parametrize("joins", [True, False])
def test_launch_knobs(eng, cfg, joins):
    w = _w("between_across_2^32", joins)
    want = oracle.run_query(w, from_encoded=False, threads=0)
    t = dpf.Tuning(cfg.get("chunk_rows", 0), cfg.get("threads", 0), cfg.get("ht_placement", 0),
                   cfg.get("ctas_per_sm", 0), cfg.get("staging", 0), 0)
    assert_same(eng.run(w, tuning=t), want, cfg)


def test_host_resident_pages():
    w = _w("two_ranges", True, rows=(1 << 19) + 77, seed=8)
    e = dpf.Engine(device=0)
    try:
        e.load_workload(w, placement="host")
        assert_same(e.run(w), oracle.run_query(w, from_encoded=False, threads=0), "host")
    finally:
        e.close()


def test_batch_with_32_bit_plans(eng):
    """One launch over plans with and without 64-bit filters (and staging
    asked for: a batch stages all its queries or none)."""
    ws = [_w("gt_2^40", False, seed=11), synth.star_join(rows=(1 << 20) + 5, page_rows=65536, seed=12),
          _w("le_3x2^31", True, seed=13), synth.scan_filter_aggregate(rows=300000, page_rows=32768, seed=14)]
    for w in ws:
        eng.load_workload(w)
    plans = [eng.plan(w) for w in ws]
    for st in (0, 1):
        prep = eng.ctx.prepare(plans, dpf.Tuning(0, 256, 0, 0, st, 0))
        try:
            eng.ctx.launch(prep)
            for i, w in enumerate(ws):
                assert_same(eng.ctx.read_result(prep, i), oracle.run_query(w, from_encoded=False, threads=0),
                            (st, w["name"]))
        finally:
            eng.ctx.release(prep)


@pytest.mark.parametrize("case", sorted(DIM_CASES))
def test_dimension_build(case):
    w = synth.bigint_filter_star(ROWS, 9, 65536)
    if DIM_CASES[case] == "only":
        w["query"]["joins"][0]["preds"] = []
        w = with_dim_bigint(w, [{"col": "big", "op": "between", "args": [-(1 << 35), 1 << 39]}])
    else:
        w = with_dim_bigint(w, DIM_CASES[case]())
    want = oracle.run_query(w, from_encoded=False, threads=0)
    for asynchronous in (False, True):
        e = dpf.Engine(device=0)
        try:
            assert_same(e.run(w, asynchronous=asynchronous), want, (case, asynchronous))
        finally:
            e.close()


def test_full_size():
    w = synth.bigint_filter_star(1 << 25, 5, preds=[{"col": "m1", "op": "between", "args": [3 << 30, 1 << 41]}])
    e = dpf.Engine(device=0)
    try:
        assert_same(e.run(w), oracle.run_query(w, from_encoded=False, threads=0), "2^25")
    finally:
        e.close()


def test_refusals(eng):
    w = _w("gt_2^40", False)
    eng.load_workload(w)
    m1 = eng.col(w, "fact", "m1")
    with pytest.raises(dpf.DpfError) as e:
        eng.ctx.build_hash(m1)  # a FOR64 key column
    assert e.value.status == -1
    w2 = synth.bigint_filter_star(ROWS, 7, 65536, joins=False,
                                  preds=[{"col": "m1", "op": "in", "args": [1, 2]}])
    with pytest.raises(dpf.DpfError) as e:
        eng.run(w2)  # IN with more than one operand
    assert e.value.status == -1
    with pytest.raises(dpf.DpfError) as e:
        eng.run_unfused(w)
    assert e.value.status == -1
