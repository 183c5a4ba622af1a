"""Host logic of sharded runs: contiguous page-aligned row ranges per rank
and the exact merge of per-rank results.

The fused path shards by fact pages: every rank holds the dimension tables
and scans its own range of fact pages, producing int64 group results.
Integer addition is associative, so summing the ranks' records key by key
(int64 two's-complement wrap, like the accumulators themselves) gives the
records of the whole table.  No device work happens here.
"""

from __future__ import annotations

import numpy as np

from . import RECORD_DTYPE


def shard_rows(nrows, page_rows, rank, world):
    """Rows [lo, hi) of ``rank``: whole pages, split as evenly as possible."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank out of range")
    npages = (int(nrows) + page_rows - 1) // page_rows
    p0 = npages * rank // world
    p1 = npages * (rank + 1) // world
    return min(p0 * page_rows, nrows), min(p1 * page_rows, nrows)


def slice_workload(w, lo, hi):
    """The workload restricted to fact rows [lo, hi) (dimensions unchanged)."""
    f = w["fact"]
    t = dict(w["tables"][f])
    cols = {}
    for name, c in t["cols"].items():
        if c["codec"] in ("str", "fsst"):
            offs = np.asarray(c["offsets"], np.uint64)
            a, b = int(offs[lo]), int(offs[hi])
            cols[name] = {"codec": "str", "bytes": c["bytes"][a:b], "offsets": offs[lo:hi + 1] - offs[lo]}
        else:
            cols[name] = dict(c, values=c["values"][lo:hi])
    t["cols"] = cols
    t["rows"] = hi - lo
    out = dict(w)
    out["tables"] = dict(w["tables"])
    out["tables"][f] = t
    out["name"] = f"{w['name']}_rows{lo}_{hi}"
    return out


def merge_records(parts, grouped):
    """Sums per-rank records key by key; ascending key order.  An ungrouped
    query keeps exactly one record (count 0 when every rank was empty)."""
    parts = [np.asarray(p, RECORD_DTYPE) for p in parts]
    if not grouped:
        out = np.zeros(1, RECORD_DTYPE)
        for p in parts:
            for r in p:
                out["count"][0] = np.add(out["count"][0], r["count"], dtype=np.int64)
                out["val"][0] = np.add(out["val"][0], r["val"], dtype=np.int64)
        return out
    acc = {}
    for p in parts:
        for r in p:
            k = (int(r["key"][0]), int(r["key"][1]))
            c, v = acc.get(k, (np.int64(0), np.zeros(4, np.int64)))
            acc[k] = (np.add(c, r["count"], dtype=np.int64), np.add(v, r["val"], dtype=np.int64))
    out = np.zeros(len(acc), RECORD_DTYPE)
    for i, k in enumerate(sorted(acc)):
        out["key"][i] = k
        out["count"][i], out["val"][i] = acc[k]
    return out
