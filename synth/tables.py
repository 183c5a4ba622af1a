"""Seeded table generators and query descriptions for the five workloads.

A *workload* is a plain dict::

    {"name": str,
     "tables": {table_name: {"rows": int, "page_rows": int,
                             "cols": {col_name: column}}},
     "fact": table_name,
     "query": query}

where a column is either ``{"codec": "for"|"delta"|"dict", "values":
int32 ndarray}``, ``{"codec": "for64", "values": int64 ndarray}`` (a BIGINT
column) or ``{"codec": "str", "bytes": uint8 ndarray, "offsets":
uint64 ndarray of rows+1}``.  The codec names the storage encoding the
column is to be loaded with; the generator never encodes anything itself.

A *query* is a description of the SQL it stands for::

    {"preds":  [{"col": c, "op": op, "args": [...]}, ...],   # on the fact table
     "joins":  [{"fk": c, "dim": t, "key": c,
                 "preds": [...],                              # on the dimension
                 "payload": [c | {"join": s, "field": f}, ...],
                 "joins": [join, ...]}, ...],                 # optional: a chain
     "group":  [{"col": c} | {"join": j, "field": f}, ...],   # <= 2 keys
     "aggs":   [{"op": "count"} | {"op": "sum", "cols": [a]}
                | {"op": "sum_mul", "cols": [a, b]}
                | {"op": "sum_sub", "cols": [a, b]}, ...]}    # <= 4

Predicate ops: ``lt le gt ge eq ne between in prefix contains`` (``between``
is inclusive at both ends; ``prefix`` and ``contains`` take one ``bytes``
argument).  A join's own ``joins`` (same form, ``fk`` a column of its
dimension) make a chain: the dimension's rows must match them too, and a
payload item ``{"join": s, "field": f}`` carries field f of the row's match
in sub join s.

Shapes, sizes and value distributions follow the workloads the method is
evaluated on: star-schema fact tables with uniform foreign keys into small
dimensions, a dense date dimension of seven calendar years, low-cardinality
dimension attributes, Zipf-skewed dictionary keys and short strings over a
27-symbol alphabet.
"""

from __future__ import annotations

import datetime

import numpy as np

ALPHABET = np.frombuffer(b"abcdefghijklmnopqrstuvwxyz ", dtype=np.uint8)

DEFAULT_PAGE_ROWS = 65536


def _rng(seed):
    return np.random.default_rng(np.random.SeedSequence(int(seed)))


def date_keys(first=datetime.date(1992, 1, 1), days=2556):
    """yyyymmdd keys of ``days`` consecutive calendar days from ``first``."""
    out = np.empty(days, dtype=np.int32)
    d = first
    one = datetime.timedelta(days=1)
    for i in range(days):
        out[i] = d.year * 10000 + d.month * 100 + d.day
        d += one
    return out


def _int_col(values, codec="for"):
    return {"codec": codec, "values": np.ascontiguousarray(values, dtype=np.int32)}


def _sparse_distinct(rng, count, lo, hi):
    """``count`` distinct sorted int32 values drawn from a wide range [lo, hi)
    (draws with replacement, drops repeats, draws again while short)."""
    vals = np.unique(rng.integers(lo, hi, int(count * 1.05) + 64, dtype=np.int64))
    while vals.size < count:
        vals = np.unique(np.concatenate([vals, rng.integers(lo, hi, count, dtype=np.int64)]))
    return np.sort(rng.permutation(vals)[:count]).astype(np.int32)


def _distinct_values(rng, count, lo, hi):
    """``count`` distinct sorted int32 values drawn from [lo, hi)."""
    vals = rng.choice(np.arange(lo, hi, dtype=np.int64), size=count, replace=False)
    return np.sort(vals).astype(np.int32)


# ---------------------------------------------------------------------------
# Workload 1: scan - filter - aggregate over one fact table
# ---------------------------------------------------------------------------

def scan_filter_aggregate(rows=1 << 20, seed=1, page_rows=DEFAULT_PAGE_ROWS,
                          a_lt=25, b_lo=1, b_hi=3):
    """SUM(int64(c) * d) WHERE a < a_lt AND b BETWEEN b_lo AND b_hi."""
    rng = _rng(seed)
    cols = {
        "a": _int_col(rng.integers(1, 51, rows, dtype=np.int32)),
        "b": _int_col(rng.integers(1, 51, rows, dtype=np.int32)),
        "c": _int_col(rng.integers(1, 11, rows, dtype=np.int32)),
        "d": _int_col(rng.integers(900, 105001, rows, dtype=np.int32)),
    }
    query = {
        "preds": [{"col": "a", "op": "lt", "args": [a_lt]},
                  {"col": "b", "op": "between", "args": [b_lo, b_hi]}],
        "joins": [],
        "group": [],
        "aggs": [{"op": "sum_mul", "cols": ["c", "d"]}],
    }
    return {"name": f"scan_filter_aggregate_{rows}",
            "tables": {"fact": {"rows": rows, "page_rows": page_rows, "cols": cols}},
            "fact": "fact", "query": query}


# ---------------------------------------------------------------------------
# Workload 2: star join, 4 dimensions, group by (dimension attribute, year)
# ---------------------------------------------------------------------------

def _star_dimensions(rng, dim_rows=(2000, 30000, 200000), page_rows=DEFAULT_PAGE_ROWS):
    n1, n2, n3 = dim_rows
    a1_vals = _distinct_values(rng, 10, 0, 1000)
    a2_vals = _distinct_values(rng, 25, 0, 1000)
    a3_vals = _distinct_values(rng, 25, 0, 1000)
    b3_vals = _distinct_values(rng, 5, 0, 100)
    dims = {
        "dim1": {"rows": n1, "page_rows": page_rows, "cols": {
            "k": _int_col(rng.permutation(np.arange(1, n1 + 1, dtype=np.int32))),
            "A1": _int_col(a1_vals[rng.integers(0, 10, n1)], "dict"),
        }},
        "dim2": {"rows": n2, "page_rows": page_rows, "cols": {
            "k": _int_col(rng.permutation(np.arange(1, n2 + 1, dtype=np.int32))),
            "A2": _int_col(a2_vals[rng.integers(0, 25, n2)], "dict"),
        }},
        "dim3": {"rows": n3, "page_rows": page_rows, "cols": {
            "k": _int_col(rng.permutation(np.arange(1, n3 + 1, dtype=np.int32))),
            "A3": _int_col(a3_vals[rng.integers(0, 25, n3)], "dict"),
            "B3": _int_col(b3_vals[rng.integers(0, 5, n3)], "dict"),
        }},
    }
    dk = date_keys()
    perm = rng.permutation(dk.size)
    dims["date"] = {"rows": int(dk.size), "page_rows": page_rows, "cols": {
        "k": _int_col(dk[perm]),
        "year": _int_col((dk[perm] // 10000).astype(np.int32), "dict"),
    }}
    attrs = {"A1": a1_vals, "A2": a2_vals, "A3": a3_vals, "B3": b3_vals}
    return dims, attrs


def _star_query(rng, attrs):
    v1 = int(attrs["A1"][rng.integers(0, attrs["A1"].size)])
    v2 = int(attrs["A2"][rng.integers(0, attrs["A2"].size)])
    i3 = int(rng.integers(0, attrs["A3"].size - 1))
    return {
        "preds": [],
        "joins": [
            {"fk": "fk1", "dim": "dim1", "key": "k",
             "preds": [{"col": "A1", "op": "eq", "args": [v1]}], "payload": []},
            {"fk": "fk2", "dim": "dim2", "key": "k",
             "preds": [{"col": "A2", "op": "eq", "args": [v2]}], "payload": []},
            {"fk": "fk3", "dim": "dim3", "key": "k",
             "preds": [{"col": "A3", "op": "in",
                        "args": [int(attrs["A3"][i3]), int(attrs["A3"][i3 + 1])]}],
             "payload": ["B3"]},
            {"fk": "fkd", "dim": "date", "key": "k", "preds": [], "payload": ["year"]},
        ],
        "group": [{"join": 2, "field": 0}, {"join": 3, "field": 0}],
        "aggs": [{"op": "sum", "cols": ["m1"]}],
    }


def star_join(rows=1 << 26, seed=2, page_rows=DEFAULT_PAGE_ROWS, clustered=True,
              dim_rows=(2000, 30000, 200000), date_year=None, bigint_measure=False):
    """Fact table with 4 uniform foreign keys and 2 measures, 4 dimensions.

    Filters three dimensions (10 %, 4 %, 8 %), joins all four and groups by
    (dim3.B3, date.year) computing SUM(int64 m1).  With ``clustered`` the
    fact rows are ordered by date key (a sorted load) and the date key is
    stored delta-coded; otherwise it is stored frame-of-reference coded.
    ``date_year`` adds a filter keeping one year of the date dimension.
    ``bigint_measure`` stores the measure as a BIGINT (FOR64) column holding
    m1 x 2^20 + m2 (values up to about 2^43).
    """
    rng = _rng(seed)
    dims, attrs = _star_dimensions(rng, dim_rows, page_rows)
    dk = np.sort(dims["date"]["cols"]["k"]["values"])
    n1, n2, n3 = dim_rows
    fk1 = rng.integers(1, n1 + 1, rows, dtype=np.int32)
    fk2 = rng.integers(1, n2 + 1, rows, dtype=np.int32)
    fk3 = rng.integers(1, n3 + 1, rows, dtype=np.int32)
    fkd = dk[rng.integers(0, dk.size, rows)]
    m1 = rng.integers(1, 10_000_000, rows, dtype=np.int32)
    m2 = rng.integers(1, 100_000, rows, dtype=np.int32)
    if clustered:
        order = np.argsort(fkd, kind="stable")
        fk1, fk2, fk3, fkd, m1, m2 = (x[order] for x in (fk1, fk2, fk3, fkd, m1, m2))
    fact = {"rows": rows, "page_rows": page_rows, "cols": {
        "fk1": _int_col(fk1), "fk2": _int_col(fk2), "fk3": _int_col(fk3),
        "fkd": _int_col(fkd, "delta" if clustered else "for"),
        "m1": _int_col(m1), "m2": _int_col(m2),
    }}
    if bigint_measure:
        fact["cols"]["m1"] = {"codec": "for64", "values": (m1.astype(np.int64) << 20) + m2}
    tables = dict(dims)
    tables["fact"] = fact
    query = _star_query(rng, attrs)
    name = f"star_join_{rows}{'_clustered' if clustered else ''}{'_bigint' if bigint_measure else ''}"
    if date_year is not None:
        # one year of the date dimension (an SSB Q1/Q3-style date filter);
        # the fact tables are the same as without it
        query["joins"][3]["preds"] = [{"col": "year", "op": "eq", "args": [int(date_year)]}]
    return {"name": name, "tables": tables, "fact": "fact", "query": query}


# ---------------------------------------------------------------------------
# Workload 2b: a chain of joins, LINEITEM -> ORDERS -> CUSTOMER
# ---------------------------------------------------------------------------

def chain_join(rows=1 << 26, seed=5, page_rows=DEFAULT_PAGE_ROWS, orders_per_row=0.25,
               customers_per_order=0.1, sparse_orderkeys=False, segment=None):
    """Three tables shaped like TPC-H's LINEITEM, ORDERS and CUSTOMER.

    ORDERS has ``rows * orders_per_row`` rows with unique order keys drawn
    from [1, 4 x orders] (TPC-H uses a quarter of its key space), uniform
    customer keys, order dates over the seven-year date range and five
    priorities.  CUSTOMER has ``orders * customers_per_order`` rows with
    five market segments and 25 nations.  LINEITEM rows are sorted by order
    key (about four per order, Poisson) and stored delta-coded, as a table
    loaded in order-key order would be; ship dates fall 1..121 days after
    the order date.  With ``sparse_orderkeys`` the order keys spread over
    the positive int32 range (an open-addressing ORDERS table).

    The query (TPC-H Q3-shaped, grouped on small keys):
        SELECT c_nation, o_priority, COUNT(*), SUM(l_price),
               SUM(l_price * l_discount)
        FROM lineitem JOIN orders ON l_orderkey = o_orderkey
                      JOIN customer ON o_custkey = c_custkey
        WHERE c_segment = S AND o_orderdate < D AND l_shipdate > D
        GROUP BY c_nation, o_priority
    as a chain: CUSTOMER's table is probed by the ORDERS scan, whose table
    carries c_nation and o_priority to the LINEITEM scan.
    """
    rng = _rng(seed)
    n_orders = max(int(rows * orders_per_row), 1)
    n_cust = max(int(n_orders * customers_per_order), 1)
    dk = date_keys()
    seg_vals = _distinct_values(rng, 5, 0, 100)
    nation_vals = np.arange(25, dtype=np.int32)
    customer = {"rows": n_cust, "page_rows": page_rows, "cols": {
        "c_custkey": _int_col(rng.permutation(np.arange(1, n_cust + 1, dtype=np.int32))),
        "c_segment": _int_col(seg_vals[rng.integers(0, 5, n_cust)], "dict"),
        "c_nation": _int_col(nation_vals[rng.integers(0, 25, n_cust)], "dict"),
    }}
    if sparse_orderkeys:
        okeys = _sparse_distinct(rng, n_orders, 1, 2**31 - 1)
    else:
        okeys = np.sort(rng.choice(np.arange(1, 4 * n_orders + 1, dtype=np.int32), n_orders, replace=False))
    n_orders = int(okeys.size)
    o_date_idx = rng.integers(0, dk.size - 151, n_orders)
    prio_vals = np.arange(1, 6, dtype=np.int32)
    operm = rng.permutation(n_orders)  # ORDERS is not stored in key order
    orders = {"rows": n_orders, "page_rows": page_rows, "cols": {
        "o_orderkey": _int_col(okeys[operm]),
        "o_custkey": _int_col(rng.integers(1, n_cust + 1, n_orders, dtype=np.int32)),
        "o_orderdate": _int_col(dk[o_date_idx[operm]]),
        "o_priority": _int_col(prio_vals[rng.integers(0, 5, n_orders)], "dict"),
    }}
    l_idx = np.sort(rng.integers(0, n_orders, rows).astype(np.int32))
    lineitem = {"rows": rows, "page_rows": page_rows, "cols": {
        "l_orderkey": _int_col(okeys[l_idx], "delta"),
        "l_shipdate": _int_col(dk[o_date_idx[l_idx] + rng.integers(1, 122, rows)]),
        "l_price": _int_col(rng.integers(90_000, 10_500_001, rows, dtype=np.int32)),
        "l_discount": _int_col(rng.integers(0, 11, rows, dtype=np.int32)),
    }}
    seg = int(seg_vals[int(rng.integers(0, 5))] if segment is None else segment)
    cut = int(dk[int(dk.size * 0.45)])  # about 1995-03-15, as in TPC-H Q3
    query = {
        "preds": [{"col": "l_shipdate", "op": "gt", "args": [cut]}],
        "joins": [{"fk": "l_orderkey", "dim": "orders", "key": "o_orderkey",
                   "preds": [{"col": "o_orderdate", "op": "lt", "args": [cut]}],
                   "payload": [{"join": 0, "field": 0}, "o_priority"],
                   "joins": [{"fk": "o_custkey", "dim": "customer", "key": "c_custkey",
                              "preds": [{"col": "c_segment", "op": "eq", "args": [seg]}],
                              "payload": ["c_nation"]}]}],
        "group": [{"join": 0, "field": 0}, {"join": 0, "field": 1}],
        "aggs": [{"op": "count"}, {"op": "sum", "cols": ["l_price"]},
                 {"op": "sum_mul", "cols": ["l_price", "l_discount"]}],
    }
    name = f"chain_join_{rows}{'_sparse' if sparse_orderkeys else ''}"
    return {"name": name, "tables": {"customer": customer, "orders": orders, "lineitem": lineitem},
            "fact": "lineitem", "query": query}


def bigint_filter_star(rows=1 << 16, seed=7, page_rows=DEFAULT_PAGE_ROWS, preds=None, joins=True):
    """The star join with its measure m1 stored as a BIGINT (FOR64) column
    (m1 x 2^20 + m2, values up to about 2^43) and predicates on that
    measure, so bounds above and below 2^32 are compared in 64 bits.
    ``preds`` defaults to m1 BETWEEN 2^35 AND 2^42.  With ``joins=False``
    the joins and group keys are dropped and only the fact table is kept:
    the 64-bit predicates are then the plan's only filters (COUNT(*) and
    SUM(m1) over the fact alone)."""
    w = star_join(rows, seed, page_rows, clustered=False, bigint_measure=True)
    q = w["query"]
    q["preds"] = list(preds) if preds is not None else [{"col": "m1", "op": "between", "args": [1 << 35, 1 << 42]}]
    if not joins:
        q["joins"] = []
        q["group"] = []
        q["aggs"] = [{"op": "count"}, {"op": "sum", "cols": ["m1"]}]
        w["tables"] = {"fact": w["tables"]["fact"]}
    w["name"] = f"star_bigint_filter_{rows}_{seed}{'' if joins else '_alone'}"
    return w


def tiny_chain_workload(seed, rows=None, page_rows=None, max_dim_rows=None):
    """A random small chain (fact -> mid -> leaf, sometimes -> leaf2 below
    leaf, sometimes a second table probed by mid) with random predicates,
    payload sources, dense or sparse keys and empty results.
    ``max_dim_rows`` caps every table below the fact (and the fact at four
    times that), for evaluators that search row by row."""
    rng = _rng(5000 + seed)
    if page_rows is None:
        page_rows = int(rng.choice([128, 256, 1024]))
    if rows is None:
        rows = int(rng.integers(1, 5 * page_rows))
    cap = (lambda n: n) if max_dim_rows is None else (lambda n: max(1, min(n, max_dim_rows)))
    if max_dim_rows is not None:
        rows = min(rows, 4 * max_dim_rows)

    def keys(n):
        if rng.integers(0, 3) == 0:  # sparse: an open-addressing table
            return rng.permutation(_sparse_distinct(rng, n, -(2**31) + 1, 2**31 - 1))
        return rng.permutation(np.arange(1, n + 1, dtype=np.int32) * int(rng.integers(1, 4)))

    def table(n, extra):
        cols = {"k": _int_col(keys(n), "for"),
                "A": _int_col(rng.integers(0, 6, n, dtype=np.int32) * 5 - 7, "dict"),
                "B": _int_col(rng.integers(0, 3, n, dtype=np.int32) + 40, "dict"),
                "x": _int_col(rng.integers(-50, 51, n, dtype=np.int32), "delta" if rng.integers(0, 2) else "for")}
        cols.update(extra)
        return {"rows": n, "page_rows": page_rows, "cols": cols}

    def fk_into(tab, n):
        k = tab["cols"]["k"]["values"]
        miss = int(k.max()) + 1 if k.max() < 2**31 - 1 else int(k.min()) - 1
        pool = np.append(k, np.int32(miss))  # one key that never matches
        return pool[rng.integers(0, pool.size, n)].astype(np.int32)

    def dpreds():
        out = []
        if rng.integers(0, 2):
            out.append({"col": "x", "op": str(rng.choice(["lt", "ge", "between"])),
                        "args": sorted(int(v) for v in rng.integers(-60, 61, 2))})
            if out[-1]["op"] != "between":
                out[-1]["args"] = out[-1]["args"][:1]
        if rng.integers(0, 3) == 0:
            out.append({"col": "A", "op": "ne", "args": [int(rng.integers(0, 6)) * 5 - 7]})
        return out

    n_leaf = cap(int(rng.integers(1, 400)))
    leaf = table(n_leaf, {})
    tables = {"leaf": leaf}
    leaf_join = {"fk": "fk_leaf", "dim": "leaf", "key": "k", "preds": dpreds(),
                 "payload": [str(c) for c in rng.choice(["A", "B"], int(rng.integers(0, 3)), replace=False)]}
    if rng.integers(0, 3) == 0:  # a deeper chain: leaf itself probes leaf2
        n2 = cap(int(rng.integers(1, 200)))
        tables["leaf2"] = table(n2, {})
        leaf["cols"]["fk_leaf2"] = _int_col(fk_into(tables["leaf2"], n_leaf), "for")
        leaf_join["joins"] = [{"fk": "fk_leaf2", "dim": "leaf2", "key": "k", "preds": dpreds(),
                               "payload": ["B"]}]
        if rng.integers(0, 2) and len(leaf_join["payload"]) < 2:
            leaf_join["payload"].append({"join": 0, "field": 0})
    n_mid = cap(int(rng.integers(1, 1500)))
    mid = table(n_mid, {"fk_leaf": _int_col(fk_into(leaf, n_mid), "delta" if rng.integers(0, 2) else "for")})
    tables["mid"] = mid
    mid_joins = [leaf_join]
    if rng.integers(0, 3) == 0:  # mid probes two tables
        n_side = cap(int(rng.integers(1, 100)))
        tables["side"] = table(n_side, {})
        mid["cols"]["fk_side"] = _int_col(fk_into(tables["side"], n_mid), "for")
        mid_joins.append({"fk": "fk_side", "dim": "side", "key": "k", "preds": dpreds(), "payload": ["A"]})
    pay_choices = [{"join": s, "field": f} for s, j in enumerate(mid_joins) for f in range(len(j["payload"]))]
    pay_choices += ["A", "B"]
    npay = int(rng.integers(0, 3))
    mid_pay = [pay_choices[i] for i in rng.choice(len(pay_choices), min(npay, len(pay_choices)), replace=False)]
    fact = {"rows": rows, "page_rows": page_rows, "cols": {
        "fk_mid": _int_col(np.sort(fk_into(mid, rows)) if rng.integers(0, 2) else fk_into(mid, rows),
                           "delta" if rng.integers(0, 2) else "for"),
        "m": _int_col(rng.integers(-1000, 1001, rows, dtype=np.int32)),
        "g": _int_col(rng.integers(0, 4, rows, dtype=np.int32), "dict"),
    }}
    tables["fact"] = fact
    preds = []
    if rng.integers(0, 2):
        preds.append({"col": "m", "op": "gt", "args": [int(rng.integers(-1000, 1001))]})
    mid_join = {"fk": "fk_mid", "dim": "mid", "key": "k", "preds": dpreds(), "payload": mid_pay,
                "joins": mid_joins}
    group = []
    for f in rng.permutation(len(mid_pay))[:int(rng.integers(0, 3))]:
        group.append({"join": 0, "field": int(f)})
    if len(group) < 2 and rng.integers(0, 2):
        group.append({"col": "g"})
    aggs = [{"op": "count"}, {"op": "sum", "cols": ["m"]}]
    query = {"preds": preds, "joins": [mid_join], "group": group, "aggs": aggs}
    return {"name": f"tiny_chain_{seed}", "tables": tables, "fact": "fact", "query": query}


# ---------------------------------------------------------------------------
# Workload 3: variable-length strings, prefix filter, Zipf dictionary key
# ---------------------------------------------------------------------------

def _zipf_codes(rng, rows, n_keys=1024, s=1.1):
    """Ranks 0..n_keys-1 with P(rank k) proportional to (k+1)^-s (inverse CDF)."""
    w = np.arange(1, n_keys + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = rng.random(rows)
    return np.minimum(np.searchsorted(cdf, u, side="right"), n_keys - 1)


def random_strings(rng, rows, min_len=10, max_len=44):
    lengths = rng.integers(min_len, max_len + 1, rows, dtype=np.int64)
    offsets = np.zeros(rows + 1, dtype=np.uint64)
    np.cumsum(lengths, out=offsets[1:])
    total = int(offsets[-1])
    data = ALPHABET[rng.integers(0, ALPHABET.size, total, dtype=np.uint8)]
    return np.ascontiguousarray(data), offsets


def text_strings(rng, rows, min_len=10, max_len=44, n_words=512):
    """Strings of words: a stream of words from a vocabulary of n_words words
    of 3..9 letters (Zipf(1.1) word frequencies), each followed by a space,
    cut into consecutive pieces of lengths drawn uniformly from
    min_len..max_len.  Text-like, so a symbol-table codec (FSST) compresses
    it, unlike uniform random bytes."""
    letters = ALPHABET[ALPHABET != ord(" ")]
    wl = rng.integers(3, 10, n_words)
    W = np.full((n_words, 10), ord(" "), dtype=np.uint8)
    for i, k in enumerate(wl):
        W[i, :k] = letters[rng.integers(0, letters.size, int(k))]
    wlen = wl + 1  # the word and its space
    w = np.arange(1, n_words + 1, dtype=np.float64) ** (-1.1)
    cdf = np.cumsum(w) / w.sum()
    lengths = rng.integers(min_len, max_len + 1, rows, dtype=np.int64)
    total = int(lengths.sum())
    need = int(total / (wlen.mean() * 0.9)) + 16
    while True:
        pick = np.minimum(np.searchsorted(cdf, rng.random(need), side="right"), n_words - 1)
        stream = W[pick][np.arange(10)[None, :] < wlen[pick][:, None]]
        if stream.size >= total:
            break
        need *= 2
    offsets = np.zeros(rows + 1, dtype=np.uint64)
    np.cumsum(lengths, out=offsets[1:])
    words = [bytes(W[i, :k]) for i, k in enumerate(wl)]
    return np.ascontiguousarray(stream[:total]), offsets, words


def strings(rows=1 << 25, seed=3, page_rows=DEFAULT_PAGE_ROWS, prefix=b"q",
            n_keys=1024, codec="str", text=False, contains=None):
    """COUNT(*), SUM(int64 m) WHERE s LIKE 'prefix%' GROUP BY key.

    ``text``: word-based strings instead of uniform random bytes; ``codec``:
    "str" (offsets + raw bytes) or "fsst"; ``contains``: the predicate
    becomes s LIKE '%contains%' (a substring anywhere)."""
    rng = _rng(seed)
    if text:
        data, offsets, _ = text_strings(rng, rows)
    else:
        data, offsets = random_strings(rng, rows)
    key_values = rng.choice(np.arange(-32768, 32768, dtype=np.int32), size=n_keys,
                            replace=False).astype(np.int32)
    key = key_values[_zipf_codes(rng, rows, n_keys)]
    m = rng.integers(1, 1_000_001, rows, dtype=np.int32)
    fact = {"rows": rows, "page_rows": page_rows, "cols": {
        "s": {"codec": codec, "bytes": data, "offsets": offsets},
        "key": _int_col(key, "dict"),
        "m": _int_col(m),
    }}
    pred = ({"col": "s", "op": "contains", "args": [bytes(contains)]} if contains is not None
            else {"col": "s", "op": "prefix", "args": [bytes(prefix)]})
    query = {
        "preds": [pred],
        "joins": [],
        "group": [{"col": "key"}],
        "aggs": [{"op": "count"}, {"op": "sum", "cols": ["m"]}],
    }
    name = (f"strings_{rows}" + ("_text" if text else "") + ("" if codec == "str" else f"_{codec}")
            + ("_all" if contains is None and not prefix else ""))
    return {"name": name, "tables": {"fact": fact}, "fact": "fact", "query": query}


# ---------------------------------------------------------------------------
# Workload 4: a batch of queries of the three shapes over uneven tables
# ---------------------------------------------------------------------------

def batched_workloads(n_queries=64, seed=4, log2_lo=16.0, log2_hi=26.0,
                      page_rows=DEFAULT_PAGE_ROWS, max_rows=None):
    """``n_queries`` workloads; shape uniform over the three above, fact rows
    round(2^U(log2_lo, log2_hi)), predicate constants drawn per query."""
    rng = _rng(seed)
    out = []
    for q in range(n_queries):
        shape = int(rng.integers(1, 4))
        rows = int(round(2.0 ** rng.uniform(log2_lo, log2_hi)))
        if max_rows is not None:
            rows = min(rows, int(max_rows))
        sub_seed = int(rng.integers(1, 2**31))
        if shape == 1:
            sub = _rng(sub_seed)
            w = scan_filter_aggregate(rows, sub_seed, page_rows,
                                      a_lt=int(sub.integers(2, 50)),
                                      b_lo=int(sub.integers(1, 10)),
                                      b_hi=int(sub.integers(10, 20)))
        elif shape == 2:
            w = star_join(rows, sub_seed, page_rows, clustered=bool(rng.integers(0, 2)))
        else:
            sub = _rng(sub_seed)
            pfx = bytes(ALPHABET[sub.integers(0, ALPHABET.size, int(sub.integers(1, 3)))])
            w = strings(rows, sub_seed, page_rows, prefix=pfx)
        w["name"] = f"q{q:02d}_{w['name']}"
        out.append(w)
    return out


def serve_variants(w, n_star=12, n_scan=4, seed=5):
    """Query variants over one resident star schema ``w`` (the serving mix):
    ``n_star`` star joins with the dimension predicate constants re-drawn
    from the dimensions' own values, then ``n_scan`` scan-filter-aggregates
    over the fact's measures (``m2 < x AND m1 BETWEEN lo AND hi``, SUM(m1),
    COUNT).  Every variant shares ``w``'s tables (no copy)."""
    import copy
    rng = _rng(seed)
    out = []
    for _ in range(n_star):
        v = copy.deepcopy({k: x for k, x in w.items() if k != "tables"})
        v["tables"] = w["tables"]
        for j in v["query"]["joins"]:
            for p in j["preds"]:
                vals = np.unique(w["tables"][j["dim"]]["cols"][p["col"]]["values"])
                p["args"] = [int(x) for x in rng.choice(vals, len(p["args"]), replace=False)]
        out.append(v)
    for _ in range(n_scan):
        v = {k: w[k] for k in ("name", "tables", "fact")}
        lo = int(rng.integers(1, 5_000_000))
        v["query"] = {"preds": [{"col": "m2", "op": "lt", "args": [int(rng.integers(1000, 100_000))]},
                                {"col": "m1", "op": "between", "args": [lo, lo + int(rng.integers(1, 5_000_000))]}],
                      "joins": [], "group": [], "aggs": [{"op": "sum", "cols": ["m1"]}, {"op": "count"}]}
        out.append(v)
    return out


def hot_groups(rows=1 << 25, n_groups=5, hot_frac=0.97, seed=6, page_rows=8192):
    """A group-by stress case: group key g (n_groups values) with one value
    taking a further hot_frac of the rows, times a 3-valued key g2; int32,
    delta-coded and BIGINT measures; SUM, SUM of a product, SUM of a BIGINT
    and SUM of a BIGINT minus an int32, over rows with b >= -900 (95 %)."""
    rng = _rng(seed)
    g = rng.integers(0, n_groups, rows).astype(np.int32)
    g[rng.random(rows) < hot_frac] = 7 % n_groups
    g2 = rng.integers(0, 3, rows).astype(np.int32) * 11 - 5
    a = rng.integers(-2**31, 2**31, rows, dtype=np.int64).astype(np.int32)
    b = rng.integers(-1000, 1000, rows).astype(np.int32)
    big = rng.integers(-2**62, 2**62, rows, dtype=np.int64) // 3
    return {"name": f"hot_{rows}_{n_groups}_{seed}", "fact": "f", "tables": {"f": {
        "rows": rows, "page_rows": page_rows, "cols": {
            "g": _int_col(g, "dict"), "g2": _int_col(g2, "dict"), "a": _int_col(a),
            "b": _int_col(b, "delta"), "big": {"codec": "for64", "values": big}}}},
        "query": {"preds": [{"col": "b", "op": "ge", "args": [-900]}], "joins": [],
                  "group": [{"col": "g"}, {"col": "g2"}],
                  "aggs": [{"op": "sum", "cols": ["a"]}, {"op": "sum_mul", "cols": ["a", "b"]},
                           {"op": "sum", "cols": ["big"]}, {"op": "sum_sub", "cols": ["big", "a"]}]}}


# ---------------------------------------------------------------------------
# Small random workloads for property tests
# ---------------------------------------------------------------------------

def tiny_random_workload(seed, rows=None, page_rows=None):
    """A random small star-join-with-strings workload mixing every operator.

    Values are drawn with ranges that exercise bit widths 0..32, negative
    numbers, ragged tails and empty results.
    """
    rng = _rng(1000 + seed)
    if page_rows is None:
        page_rows = int(rng.choice([128, 256, 1024, 4096]))
    if rows is None:
        rows = int(rng.integers(1, 6 * page_rows))
    spans = [(0, 1), (0, 2), (-5, 5), (1, 50), (-(2**31), 2**31 - 1), (900, 105001)]

    def draw(n):
        lo, hi = spans[int(rng.integers(0, len(spans)))]
        return rng.integers(lo, hi, n, dtype=np.int64, endpoint=True).astype(np.int32)

    nd = int(rng.integers(1, 300))
    dim = {"rows": nd, "page_rows": page_rows, "cols": {
        "k": _int_col(rng.permutation(np.arange(1, nd + 1, dtype=np.int32))),
        "A": _int_col(rng.integers(0, 7, nd, dtype=np.int32) * 3 - 4, "dict"),
        "B": _int_col(rng.integers(0, 4, nd, dtype=np.int32) + 100, "dict"),
    }}
    data, offsets = random_strings(rng, rows, 0, int(rng.integers(1, 12)))
    fk = rng.integers(1, nd + 2, rows, dtype=np.int32)  # nd+1 never matches
    x = draw(rows)
    y = draw(rows)
    g = rng.integers(0, 5, rows, dtype=np.int32) * 7 - 10
    clustered = bool(rng.integers(0, 2))
    if clustered:
        order = np.argsort(fk, kind="stable")
        fk, x, y, g = fk[order], x[order], y[order], g[order]
        starts = offsets[:-1][order]
        lens = (offsets[1:] - offsets[:-1])[order]
        new_off = np.zeros(rows + 1, dtype=np.uint64)
        np.cumsum(lens, out=new_off[1:])
        data = np.concatenate([data[int(s):int(s + l)] for s, l in zip(starts, lens)]
                              or [np.zeros(0, np.uint8)]).astype(np.uint8)
        offsets = new_off
    fact = {"rows": rows, "page_rows": page_rows, "cols": {
        "fk": _int_col(fk, "delta" if clustered else "for"),
        "x": _int_col(x, "for"),
        "y": _int_col(y, "delta" if rng.integers(0, 2) else "for"),
        "g": _int_col(g, "dict"),
        "s": {"codec": "str", "bytes": data, "offsets": offsets},
    }}
    ops = ["lt", "le", "gt", "ge", "eq", "ne", "between", "in"]
    preds = []
    for _ in range(int(rng.integers(0, 3))):
        col = str(rng.choice(["x", "y", "g"]))
        op = str(rng.choice(ops))
        src = fact["cols"][col]["values"]
        pick = lambda: int(src[int(rng.integers(0, rows))])  # noqa: E731
        if op == "between":
            lo, hi = sorted((pick(), pick()))
            args = [lo, hi]
        elif op == "in":
            args = [pick() for _ in range(int(rng.integers(1, 5)))]
        else:
            args = [pick()]
        preds.append({"col": col, "op": op, "args": args})
    if rng.integers(0, 2):
        plen = int(rng.integers(0, 3))
        preds.append({"col": "s", "op": "prefix",
                      "args": [bytes(ALPHABET[rng.integers(0, 27, plen)])]})
    joins = []
    group = []
    if rng.integers(0, 2):
        dpreds = []
        if rng.integers(0, 2):
            dpreds.append({"col": "A", "op": "le", "args": [int(rng.integers(-4, 15))]})
        joins.append({"fk": "fk", "dim": "dim", "key": "k", "preds": dpreds,
                      "payload": ["B", "A"]})
        if rng.integers(0, 2):
            group.append({"join": 0, "field": int(rng.integers(0, 2))})
    if rng.integers(0, 2):
        group.append({"col": "g"})
    aggs = [{"op": "count"}]
    for _ in range(int(rng.integers(0, 4))):
        op = str(rng.choice(["sum", "sum_mul", "sum_sub"]))
        cols = ["x"] if op == "sum" else [str(rng.choice(["x", "y"])), str(rng.choice(["x", "y"]))]
        aggs.append({"op": op, "cols": cols})
    # the string column's codec and the string predicate's kind come from a
    # second stream, so the draws above (and earlier seeds' tables) are unchanged
    rng2 = _rng(seed + 7919)
    if rng2.integers(0, 2):
        fact["cols"]["s"] = dict(fact["cols"]["s"], codec="fsst")
    for p in preds:
        if p["col"] == "s" and rng2.integers(0, 2):
            p["op"] = "contains"
    # a BIGINT measure (FOR64) from a third stream: spans from constant to the
    # full int64 range, used by some aggregates
    rng3 = _rng(seed + 104729)
    if rng3.integers(0, 2):
        spans64 = [(7, 7), (-5, 5), (-(2**40), 2**40), (-(2**63), 2**63 - 1), (2**50, 2**50 + 1000)]
        lo, hi = spans64[int(rng3.integers(0, len(spans64)))]
        fact["cols"]["z"] = {"codec": "for64",
                             "values": rng3.integers(lo, hi, rows, dtype=np.int64, endpoint=True)}
        for a in aggs[1:]:
            if rng3.integers(0, 2):
                a["cols"] = ["z" if rng3.integers(0, 2) else c for c in a["cols"]]
        if len(aggs) < 4 and not any("z" in a.get("cols", []) for a in aggs):
            aggs.append({"op": str(rng3.choice(["sum", "sum_mul", "sum_sub"])), "cols": ["z", "x"]})
            if aggs[-1]["op"] == "sum":
                aggs[-1]["cols"] = ["z"]
    query = {"preds": preds, "joins": joins, "group": group, "aggs": aggs}
    return {"name": f"tiny_{seed}", "tables": {"fact": fact, "dim": dim},
            "fact": "fact", "query": query}
