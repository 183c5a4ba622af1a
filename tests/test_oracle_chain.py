"""Pins of the oracle's join chains (scan, probe, build: Sec. 3.1 Kernel #2).

A chain is a join whose dimension is itself joined before its table is
built (LINEITEM -> ORDERS -> CUSTOMER).  The oracle's result is pinned by

* a chain worked by hand (tests/golden/chain_hand_worked.txt: three tiny
  tables, the derivation and the expected records);
* brute force on tiny chains: plain Python loops that, for every fact row,
  search every dimension row by row (no hashing, no sorting);
* the independent numpy evaluator (``npeval``) on random chains;
* an identity that needs no evaluator of chains at all: a chain equals the
  two-join star query over a fact table into which the middle table's
  foreign key has been copied (denormalised), evaluated by the oracle's
  already-pinned star path;
* special cases: a chain whose inner table keeps every row equals the
  plain join; an inner table that keeps nothing empties the result;
  duplicate keys in an inner table are reported.
"""

import numpy as np
import pytest

import npeval
import oracle
import synth
from _hand_worked import hand_worked_chains

RECORD_DTYPE = npeval.RECORD_DTYPE


def _same(a, b, what=""):
    assert a.shape == b.shape, (what, a, b)
    for f in ("key", "count", "val"):
        assert np.array_equal(a[f], b[f]), (what, f)


def _pred_ok(cols, p, r):
    x = int(cols[p["col"]]["values"][r])
    a = [int(v) for v in p["args"]]
    return {"lt": lambda: x < a[0], "le": lambda: x <= a[0], "gt": lambda: x > a[0],
            "ge": lambda: x >= a[0], "eq": lambda: x == a[0], "ne": lambda: x != a[0],
            "between": lambda: a[0] <= x <= a[1], "in": lambda: x in a}[p["op"]]()


def _matches(w, j, key):
    """Payload tuples of the rows of j's dimension with this key that pass
    j's predicates and match every sub join (searched row by row)."""
    t = w["tables"][j["dim"]]
    cols = t["cols"]
    out = []
    for r in range(t["rows"]):
        if int(cols[j["key"]]["values"][r]) != key:
            continue
        if not all(_pred_ok(cols, p, r) for p in j["preds"]):
            continue
        subs = []
        for s in j.get("joins", []):
            m = _matches(w, s, int(cols[s["fk"]]["values"][r]))
            if not m:
                break
            subs.append(m[0])
        else:
            out.append(tuple(subs[pc["join"]][pc["field"]] if isinstance(pc, dict)
                             else int(cols[pc]["values"][r]) for pc in j["payload"]))
    return out


def _brute(w):
    q = w["query"]
    f = w["tables"][w["fact"]]
    fc = f["cols"]
    groups = {}
    for r in range(f["rows"]):
        if not all(_pred_ok(fc, p, r) for p in q["preds"]):
            continue
        hits = []
        for j in q["joins"]:
            m = _matches(w, j, int(fc[j["fk"]]["values"][r]))
            assert len(m) <= 1, "duplicate build key"
            if not m:
                break
            hits.append(m[0])
        else:
            key = [int(fc[g["col"]]["values"][r]) if "col" in g else hits[g["join"]][g["field"]]
                   for g in q["group"]]
            key = tuple(key + [0] * (2 - len(key)))
            g = groups.setdefault(key, [0, [0, 0, 0, 0]])
            g[0] += 1
            for i, a in enumerate(q["aggs"]):
                g[1][i] += 1 if a["op"] == "count" else int(fc[a["cols"][0]]["values"][r])
    if not q["group"] and not groups:
        groups[(0, 0)] = [0, [0, 0, 0, 0]]
    out = np.zeros(len(groups), RECORD_DTYPE)
    for i, k in enumerate(sorted(groups)):
        out[i]["key"] = k
        out[i]["count"] = groups[k][0]
        out[i]["val"] = groups[k][1]
    return out


def test_hand_worked_chain():
    for w, want in hand_worked_chains():
        _same(oracle.run_query(w, from_encoded=False), want, w["name"])
        _same(oracle.run_query(w, from_encoded=True), want, w["name"])
        _same(_brute(w), want, w["name"])


@pytest.mark.parametrize("seed", range(16))
def test_chain_equals_brute_force(seed):
    w = synth.tiny_chain_workload(seed, max_dim_rows=40)
    want = _brute(w)
    _same(oracle.run_query(w, from_encoded=False), want, seed)
    _same(oracle.run_query(w, from_encoded=True), want, seed)


def test_chain_equals_numpy_evaluator():
    for seed in range(12, 60):
        w = synth.tiny_chain_workload(seed)
        _same(oracle.run_query(w, from_encoded=bool(seed % 2)), npeval.evaluate(w), seed)


@pytest.mark.parametrize("sparse", [False, True])
def test_chain_equals_denormalised_star(sparse):
    """LINEITEM -> ORDERS -> CUSTOMER equals a star over LINEITEM joined to
    ORDERS and, through a copied customer key, to CUSTOMER."""
    w = synth.chain_join(rows=1 << 15, seed=9, page_rows=4096, sparse_orderkeys=sparse)
    t = w["tables"]
    ok = t["orders"]["cols"]["o_orderkey"]["values"]
    ck = t["orders"]["cols"]["o_custkey"]["values"]
    pos = {int(k): i for i, k in enumerate(ok)}
    lk = t["lineitem"]["cols"]["l_orderkey"]["values"]
    t["lineitem"]["cols"]["l_custkey"] = {"codec": "for",
                                          "values": ck[[pos[int(k)] for k in lk]].astype(np.int32)}
    chain = w["query"]["joins"][0]
    star = dict(w)
    star["query"] = dict(w["query"])
    cust = dict(chain["joins"][0], fk="l_custkey")
    orders = {k: v for k, v in chain.items() if k != "joins"}
    orders["payload"] = ["o_priority"]
    star["query"]["joins"] = [orders, cust]
    star["query"]["group"] = [{"join": 1, "field": 0}, {"join": 0, "field": 0}]
    want = oracle.run_query(star, from_encoded=False)
    got = oracle.run_query(w, from_encoded=True)
    assert want.shape[0] > 10
    _same(got, want)


def test_inner_table_keeping_everything_is_the_plain_join():
    w = synth.chain_join(rows=1 << 14, seed=3, page_rows=2048)
    j = w["query"]["joins"][0]
    j["joins"][0]["preds"] = []
    plain = dict(w, query=dict(w["query"], joins=[dict(j, joins=[], payload=["o_priority"])],
                               group=[{"join": 0, "field": 0}]))
    chain = dict(w, query=dict(w["query"], joins=[dict(j, payload=["o_priority"])],
                               group=[{"join": 0, "field": 0}]))
    _same(oracle.run_query(chain), oracle.run_query(plain))


def test_inner_table_keeping_nothing_empties_the_result():
    w = synth.chain_join(rows=1 << 14, seed=4, page_rows=2048)
    w["query"]["joins"][0]["joins"][0]["preds"] = [{"col": "c_segment", "op": "eq", "args": [-12345]}]
    assert oracle.run_query(w).shape == (0,)
    w["query"]["group"] = []
    r = oracle.run_query(w)
    assert r.shape == (1,) and r["count"][0] == 0 and not r["val"].any()


def test_duplicate_key_in_inner_table_is_reported():
    w = synth.chain_join(rows=1 << 12, seed=6, page_rows=1024)
    ck = w["tables"]["customer"]["cols"]["c_custkey"]["values"]
    ck[1] = ck[0]
    w["query"]["joins"][0]["joins"][0]["preds"] = []
    with pytest.raises(RuntimeError):
        oracle.run_query(w)
