"""Host logic of the Python engine, on CPU with a recording stand-in for the
library context: how a query description's joins become hash builds.

A join without joins of its own is one scan + build call; a join with joins
(a chain) has its inner tables built first, then one scan + probe + build
call that probes them, with payload items naming either a column of its
table or a field of one of its probed tables.  Builds are cached per
workload and join description, so a plan reuses the tables of an earlier
plan of the same query.
"""

import synth
from paper_2605_10511_gb300.engine import Engine


class RecordingCtx:
    """Records the build calls the engine makes; returns new table ids."""

    def __init__(self):
        self.calls = []
        self.next_col = 1
        self.next_ht = 100

    def load_column(self, col, table=0, page_rows=0, placement="device"):
        self.next_col += 1
        return self.next_col

    def build_hash(self, key_col, payload_cols=(), preds=(), stream=None):
        self.next_ht += 1
        self.calls.append(("build", key_col, list(payload_cols), len(preds), self.next_ht))
        return self.next_ht

    def build_hash_probe(self, key_col, payload=(), preds=(), joins=(), stream=None):
        self.next_ht += 1
        self.calls.append(("probe_build", key_col, list(payload), len(preds), list(joins), self.next_ht))
        return self.next_ht

    def build_hash_async(self, key_col, payload=(), preds=(), joins=(), stream=None):
        self.next_ht += 1
        self.calls.append(("async", key_col, list(payload), len(preds), list(joins), self.next_ht))
        return self.next_ht

    def build_hash_deferred(self, key_col, payload=(), preds=(), joins=()):
        self.next_ht += 1
        self.calls.append(("deferred", key_col, list(payload), len(preds), list(joins), self.next_ht))
        return self.next_ht

    def prepare_chain(self, builds, plans, tuning=None):
        self.calls.append(("chain", list(builds), len(plans)))
        return 7

    def close(self):
        pass


def _engine(w):
    ctx = RecordingCtx()
    eng = Engine(ctx=ctx)
    eng.load_workload(w)
    return eng, ctx


def test_chain_builds_inner_table_first_and_probes_it():
    w = synth.chain_join(rows=1 << 12, page_rows=1024)
    eng, ctx = _engine(w)
    hts = eng.build_joins(w)
    assert [c[0] for c in ctx.calls] == ["build", "probe_build"]
    cust, orders = ctx.calls
    # CUSTOMER: key c_custkey, payload c_nation, one predicate (segment)
    assert cust[1] == eng.col(w, "customer", "c_custkey")
    assert cust[2] == [eng.col(w, "customer", "c_nation")]
    assert cust[3] == 1
    # ORDERS: key o_orderkey; payload (field 0 of join 0, o_priority); one
    # predicate (date); one join probing CUSTOMER's table through o_custkey
    assert orders[1] == eng.col(w, "orders", "o_orderkey")
    assert orders[2] == [("join", 0, 0), eng.col(w, "orders", "o_priority")]
    assert orders[3] == 1
    assert orders[4] == [(eng.col(w, "orders", "o_custkey"), cust[4])]
    assert hts == [orders[5]]


def test_builds_are_cached_per_join_description():
    w = synth.chain_join(rows=1 << 12, page_rows=1024)
    eng, ctx = _engine(w)
    first = eng.build_joins(w)
    n = len(ctx.calls)
    assert eng.build_joins(w) == first and len(ctx.calls) == n
    # another predicate constant on the inner table is another chain: both
    # tables are built again (the outer one probes the new inner table)
    w2 = dict(w)
    w2["query"] = {**w["query"], "joins": [dict(w["query"]["joins"][0])]}
    inner = dict(w2["query"]["joins"][0]["joins"][0])
    inner["preds"] = [{"col": "c_segment", "op": "ne", "args": [inner["preds"][0]["args"][0]]}]
    w2["query"]["joins"][0]["joins"] = [inner]
    eng.build_joins(w2)
    assert [c[0] for c in ctx.calls[n:]] == ["build", "probe_build"]
    assert ctx.calls[-1][4][0][1] == ctx.calls[-2][4]


def test_deeper_chains_and_two_probed_tables():
    seen = {"depth3": False, "two_probed": False, "carried": False}
    for seed in range(60):
        w = synth.tiny_chain_workload(seed)
        eng, ctx = _engine(w)
        eng.build_joins(w)
        mid = w["query"]["joins"][0]
        subs = mid["joins"]
        probe_builds = [c for c in ctx.calls if c[0] == "probe_build"]
        # the outermost table's build is the last call and probes one table per sub join
        assert ctx.calls[-1][0] == "probe_build" and len(ctx.calls[-1][4]) == len(subs)
        if any(s.get("joins") for s in subs):
            seen["depth3"] = True
            assert len(probe_builds) == 2  # leaf (probing leaf2), then mid
        if len(subs) == 2:
            seen["two_probed"] = True
        if any(isinstance(p, dict) for p in mid["payload"]):
            seen["carried"] = True
            assert any(isinstance(p, tuple) and p[0] == "join" for p in ctx.calls[-1][2])
        # every table a build probes was built by an earlier call
        made = set()
        for c in ctx.calls:
            if c[0] == "probe_build":
                assert all(ht in made for _, ht in c[4])
            made.add(c[-1])
    assert all(seen.values()), seen


def test_plain_joins_use_the_scan_and_build_call():
    w = synth.star_join(rows=1 << 12, page_rows=1024, dim_rows=(200, 300, 400))
    eng, ctx = _engine(w)
    eng.build_joins(w)
    assert [c[0] for c in ctx.calls] == ["build"] * 4


def test_enqueue_only_and_deferred_builds_route_every_table():
    """With ``asynchronous`` or ``deferred`` every table of a chain, the
    inner one included, goes through the scan + probe + build form of that
    mode (a table without joins is the same call with no joins); deferred
    tables are kept apart from built ones, and a prepared chain names them
    inner first."""
    w = synth.chain_join(rows=1 << 12, page_rows=1024)
    for mode in ("async", "deferred"):
        eng, ctx = _engine(w)
        hts = eng.build_joins(w, asynchronous=mode == "async", deferred=mode == "deferred")
        assert [c[0] for c in ctx.calls] == [mode, mode]
        cust, orders = ctx.calls
        assert cust[1] == eng.col(w, "customer", "c_custkey") and cust[4] == []
        assert cust[2] == [eng.col(w, "customer", "c_nation")]
        assert orders[4] == [(eng.col(w, "orders", "o_custkey"), cust[5])]
        assert hts == [orders[5]]
        assert eng.chain_tables(w, deferred=mode == "deferred") == [cust[5], orders[5]]
        if mode == "deferred":
            assert eng.hts == {}  # built tables untouched
            assert eng.prepare_chain(w) == 7
            assert ctx.calls[-1] == ("chain", [cust[5], orders[5]], 1)
            assert [c[0] for c in ctx.calls[:-1]] == ["deferred", "deferred"]  # the plan reused them
