"""Pins of the oracle's predicates on BIGINT (FOR64) columns (CPU only).

Sec. 3.4.1 / Sec. 4.1 store BIGINT as 64-bit GPU-FOR.  A predicate on such a
column compares the int64 value with int64 operands.  The oracle, run on
the raw arrays and on its own encoded-then-decoded pages, must give the
same records as the independent numpy evaluator (``npeval``: int64 masks)
for bounds below, across and above 2^32, for each comparison, for empty
and full selections, with the 64-bit predicate after the star's joins and
as a plan's only filter.
"""

import numpy as np
import pytest

import npeval
import synth

ROWS = 20000  # 4096-row pages: four full pages and a ragged one


def _records_equal(a, b):
    assert a.shape == b.shape, (a, b)
    for f in ("key", "count", "val"):
        assert np.array_equal(a[f], b[f]), (f, a[f], b[f])


def _value(row, seed=7):
    return int(synth.bigint_filter_star(ROWS, seed, 4096)["tables"]["fact"]["cols"]["m1"]["values"][row])


CASES = {
    "between_across_2^32": lambda: [{"col": "m1", "op": "between", "args": [3 << 30, 1 << 41]}],
    "gt_2^40": lambda: [{"col": "m1", "op": "gt", "args": [1 << 40]}],
    "le_3x2^31": lambda: [{"col": "m1", "op": "le", "args": [3 << 31]}],
    "lt_2^42": lambda: [{"col": "m1", "op": "lt", "args": [1 << 42]}],
    "ge_2^43": lambda: [{"col": "m1", "op": "ge", "args": [1 << 43]}],
    "eq_a_value": lambda: [{"col": "m1", "op": "eq", "args": [_value(5)]}],
    "ne_a_value": lambda: [{"col": "m1", "op": "ne", "args": [_value(5)]}],
    "in_one_value": lambda: [{"col": "m1", "op": "in", "args": [_value(11)]}],
    "empty": lambda: [{"col": "m1", "op": "lt", "args": [0]}],
    "all": lambda: [{"col": "m1", "op": "ge", "args": [-(1 << 62)]}],
    "two_ranges": lambda: [{"col": "m1", "op": "gt", "args": [1 << 36]},
                           {"col": "m1", "op": "le", "args": [(1 << 42) + 12345]}],
}


@pytest.mark.parametrize("joins", [True, False])
@pytest.mark.parametrize("case", sorted(CASES))
def test_oracle_matches_numpy(oracle_lib, case, joins):
    w = synth.bigint_filter_star(ROWS, 7, 4096, preds=CASES[case](), joins=joins)
    want = npeval.evaluate(w)
    _records_equal(oracle_lib.run_query(w, from_encoded=False), want)
    _records_equal(oracle_lib.run_query(w, from_encoded=True), want)


def test_bounds_cut_values_above_2_32(oracle_lib):
    """The generated measure spans beyond 2^32, so truncating either side to
    32 bits would change these counts."""
    v = synth.bigint_filter_star(ROWS, 7, 4096)["tables"]["fact"]["cols"]["m1"]["values"]
    assert v.max() > 1 << 40 and v.min() < 1 << 32
    w = synth.bigint_filter_star(ROWS, 7, 4096, preds=[{"col": "m1", "op": "gt", "args": [1 << 40]}],
                                 joins=False)
    got = oracle_lib.run_query(w, from_encoded=True)
    assert int(got["count"][0]) == int((v > (1 << 40)).sum())
    assert int(got["val"][0][0]) == int((v > (1 << 40)).sum())  # the COUNT aggregate
    assert int(got["val"][0][1]) == int(v[v > (1 << 40)].sum())


def with_dim_bigint(w, preds, seed=3):
    """w with a BIGINT column ``big`` (values up to about 2^41) added to
    dim1 and ``preds`` on it added to dim1's build predicates."""
    rng = np.random.default_rng(seed)
    d = w["tables"]["dim1"]
    d["cols"]["big"] = {"codec": "for64",
                        "values": rng.integers(-(1 << 40), 1 << 41, d["rows"], dtype=np.int64)}
    j = w["query"]["joins"][0]
    j["preds"] = list(j["preds"]) + list(preds)
    return w


DIM_CASES = {
    "with_a_32_bit_predicate": lambda: [{"col": "big", "op": "gt", "args": [0]}],
    "only_64_bit": "only",
    "ne": lambda: [{"col": "big", "op": "ne", "args": [7]}],
}


@pytest.mark.parametrize("case", sorted(DIM_CASES))
def test_dimension_build_with_a_bigint_predicate(oracle_lib, case):
    w = synth.bigint_filter_star(ROWS, 9, 4096)
    if DIM_CASES[case] == "only":
        w["query"]["joins"][0]["preds"] = []
        w = with_dim_bigint(w, [{"col": "big", "op": "between", "args": [-(1 << 35), 1 << 39]}])
    else:
        w = with_dim_bigint(w, DIM_CASES[case]())
    want = npeval.evaluate(w)
    _records_equal(oracle_lib.run_query(w, from_encoded=False), want)
    _records_equal(oracle_lib.run_query(w, from_encoded=True), want)
