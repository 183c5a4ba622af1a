"""Loads workload tables into a library context and turns query descriptions
into plans (argument marshalling only; the work is done by the library).

A query description has the form documented in ``synth.tables``: fact
predicates, equi-joins against dimension tables (with dimension predicates,
payload columns and, for a chain, joins of the dimension itself), up to two
group keys and up to four aggregates.
"""

from __future__ import annotations

import ctypes as C

from . import AGG, Agg, Context, Join, Key, Plan, Pred, make_pred


class PlanHandle:
    """A ``dpf_plan`` plus the ctypes arrays it points into."""

    def __init__(self, plan, keep):
        self.plan = plan
        self._keep = keep


class Engine:
    def __init__(self, device=0, hbm_budget=0, use_torch_allocator=False, ctx=None):
        self.ctx = ctx or Context(device, hbm_budget, use_torch_allocator)
        self.cols = {}       # (workload name, table, column) -> column id
        self.tables = {}     # (workload name, table) -> table id
        self.hts = {}        # join signature -> hash table id
        self.dhts = {}       # join signature -> deferred hash table id (prepared chains)

    def close(self):
        self.ctx.close()

    # ------------------------------------------------------------------ loading
    def load_workload(self, w, placement="device", fact_placement=None):
        """Loads every column of every table of workload ``w`` (once)."""
        for tname, t in w["tables"].items():
            key = (w["name"], tname)
            if key in self.tables:
                continue
            tid = len(self.tables) + 1
            self.tables[key] = tid
            place = fact_placement if (fact_placement and tname == w["fact"]) else placement
            for cname, c in t["cols"].items():
                self.cols[(w["name"], tname, cname)] = self.ctx.load_column(
                    c, table=tid, page_rows=t["page_rows"], placement=place)

    def col(self, w, table, name):
        return self.cols[(w["name"], table, name)]

    def fact_bytes(self, w):
        """Encoded bytes of every fact column the query reads (algorithmic
        bytes of one scan) and the fact row count."""
        q = w["query"]
        names = {p["col"] for p in q["preds"]} | {j["fk"] for j in q["joins"]}
        names |= {g["col"] for g in q["group"] if "col" in g}
        for a in q["aggs"]:
            names |= set(a.get("cols", []))
        total = sum(self.ctx.column_info(self.col(w, w["fact"], n))["encoded_bytes"] for n in names)
        return total, w["tables"][w["fact"]]["rows"]

    # ------------------------------------------------------------------ planning
    def build_join(self, w, j, stream=None, asynchronous=False, deferred=False):
        """Builds (or reuses) the hash table of join ``j``.  A join with
        joins of its own (a chain) has those built first; its table is then
        built by scanning its dimension and probing theirs.  With
        ``asynchronous`` every table of the chain is only enqueued on
        ``stream`` (``dpf_build_hash_async``); with ``deferred`` it is
        prepared, empty, for a prepared chain (``dpf_build_hash_deferred``,
        kept apart from the built tables)."""
        sig = (w["name"], repr(j))
        cache = self.dhts if deferred else self.hts
        if sig not in cache:
            d = j["dim"]
            preds = [make_pred(self.col(w, d, p["col"]), p["op"], p["args"]) for p in j["preds"]]
            subs = j.get("joins", [])
            if not subs and not asynchronous and not deferred and all(isinstance(c, str) for c in j["payload"]):
                pay = [self.col(w, d, c) for c in j["payload"]]
                cache[sig] = self.ctx.build_hash(self.col(w, d, j["key"]), pay, preds, stream)
            else:
                sub_hts = [(self.col(w, d, s["fk"]), self.build_join(w, s, stream, asynchronous, deferred))
                           for s in subs]
                pay = [("join", c["join"], c["field"]) if isinstance(c, dict) else self.col(w, d, c)
                       for c in j["payload"]]
                key = self.col(w, d, j["key"])
                if deferred:
                    cache[sig] = self.ctx.build_hash_deferred(key, pay, preds, sub_hts)
                else:
                    build = self.ctx.build_hash_async if asynchronous else self.ctx.build_hash_probe
                    cache[sig] = build(key, pay, preds, sub_hts, stream)
        return cache[sig]

    def build_joins(self, w, stream=None, asynchronous=False, deferred=False):
        """Builds (or reuses) the hash table of every join of ``w``'s query."""
        return [self.build_join(w, j, stream, asynchronous, deferred) for j in w["query"]["joins"]]

    def chain_tables(self, w, deferred=False):
        """Table ids of ``w``'s joins, inner tables first."""
        cache = self.dhts if deferred else self.hts
        out = []

        def walk(j):
            for s in j.get("joins", []):
                walk(s)
            out.append(cache[(w["name"], repr(j))])
        for j in w["query"]["joins"]:
            walk(j)
        return out

    def prepare_chain(self, w, tuning=None):
        """``w``'s query as one prepared chain: deferred tables for every join
        (inner first) and the plan over them; every launch of the returned
        batch rebuilds the tables and runs the plan."""
        self.load_workload(w)
        h = self.plan(w, deferred=True)
        return self.ctx.prepare_chain(self.chain_tables(w, deferred=True), [h], tuning)

    def plan(self, w, stream=None, asynchronous=False, deferred=False):
        q = w["query"]
        f = w["fact"]
        hts = self.build_joins(w, stream, asynchronous, deferred)
        preds = (Pred * max(len(q["preds"]), 1))(
            *[make_pred(self.col(w, f, p["col"]), p["op"], p["args"]) for p in q["preds"]])
        joins = (Join * max(len(q["joins"]), 1))(
            *[Join(self.col(w, f, j["fk"]), h) for j, h in zip(q["joins"], hts)])
        keys = (Key * max(len(q["group"]), 1))()
        for i, g in enumerate(q["group"]):
            if "col" in g:
                keys[i] = Key(0, self.col(w, f, g["col"]), 0, 0)
            else:
                keys[i] = Key(1, 0, g["join"], g["field"])
        aggs = (Agg * max(len(q["aggs"]), 1))()
        for i, a in enumerate(q["aggs"]):
            cols = [self.col(w, f, c) for c in a.get("cols", [])]
            aggs[i] = Agg(AGG[a["op"]], cols[0] if cols else 0, cols[1] if len(cols) > 1 else 0)
        plan = Plan(len(q["preds"]), C.cast(preds, C.POINTER(Pred)),
                    len(q["joins"]), C.cast(joins, C.POINTER(Join)),
                    len(q["group"]), C.cast(keys, C.POINTER(Key)),
                    len(q["aggs"]), C.cast(aggs, C.POINTER(Agg)),
                    self.col(w, f, next(iter(w["tables"][f]["cols"]))))
        return PlanHandle(plan, (preds, joins, keys, aggs))

    def run(self, w, stream=None, tuning=None, asynchronous=False):
        """Loads (if needed), plans, launches and reads one query's records
        (with ``asynchronous``, its tables are built by enqueue-only builds
        on ``stream``, checked by ``hash_wait`` after the records are read)."""
        self.load_workload(w)
        h = self.plan(w, stream, asynchronous)
        prep = self.ctx.prepare([h], tuning)
        try:
            self.ctx.launch(prep, stream)
            rec = self.ctx.read_result(prep, 0)
        finally:
            self.ctx.release(prep)
        if asynchronous:
            self.wait_joins(w)
        return rec

    def wait_joins(self, w, deferred=False):
        """``hash_wait`` on every table of ``w``'s query, inner tables first
        (raises the first build error)."""
        for ht in self.chain_tables(w, deferred):
            self.ctx.hash_wait(ht)

    def run_unfused(self, w, stream=None):
        """The same query through the unfused per-operator chain."""
        self.load_workload(w)
        h = self.plan(w, stream)
        prep = self.ctx.prepare_unfused(h)
        try:
            self.ctx.launch(prep, stream)
            return self.ctx.read_result(prep, 0)
        finally:
            self.ctx.release(prep)
