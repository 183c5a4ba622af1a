"""An independent numpy evaluator of the query definition, used to pin the oracle.

It reads the raw generated arrays (never any encoded page) and evaluates the
same SQL with vectorised library routines: boolean masks for predicates,
``np.searchsorted`` over the sorted build keys for the equi-joins (applied
recursively to a dimension that is itself joined: a chain),
``np.unique(..., return_inverse=True)`` for grouping and ``np.add.at`` /
``np.bincount`` for the int64 aggregates.  It shares nothing with the C++
oracle beyond the query description.
"""

import numpy as np

RECORD_DTYPE = np.dtype([("key", np.int32, (2,)), ("count", np.int64), ("val", np.int64, (4,))])


def _pred_mask(cols, pred, n):
    op, args = pred["op"], pred["args"]
    c = cols[pred["col"]]
    if op == "prefix":
        pfx = np.frombuffer(bytes(args[0]), dtype=np.uint8)
        data, offs = c["bytes"], c["offsets"].astype(np.int64)
        lens = offs[1:] - offs[:-1]
        ok = lens >= pfx.size
        for i in range(pfx.size):
            idx = np.where(ok, offs[:-1] + i, 0)
            ok &= (data[idx] == pfx[i]) if data.size else np.zeros(n, bool)
        return ok
    if op == "like":
        # SQL LIKE as a regular expression ('%' -> any run, '_' -> any byte)
        # matched over the whole string by Python's own regex engine
        import re
        pat = bytes(args[0])
        rx = re.compile(b"".join(b".*" if ch == 0x25 else b"." if ch == 0x5F else re.escape(bytes([ch]))
                                 for ch in pat), re.DOTALL)
        data, offs = c["bytes"], c["offsets"].astype(np.int64)
        raw = np.asarray(data, np.uint8).tobytes()
        return np.array([rx.fullmatch(raw[offs[r]:offs[r + 1]]) is not None for r in range(n)], bool)
    if op == "contains":
        # vectorised over candidate start positions: row r matches if the
        # pattern equals bytes [offs[r] + i, offs[r] + i + m) for some i
        pat = np.frombuffer(bytes(args[0]), dtype=np.uint8)
        data, offs = c["bytes"], c["offsets"].astype(np.int64)
        lens = offs[1:] - offs[:-1]
        if pat.size == 0:
            return np.ones(n, bool)
        found = np.zeros(n, bool)
        for i in range(int(lens.max(initial=0)) - pat.size + 1):
            ok = lens >= i + pat.size
            for k in range(pat.size):
                idx = np.where(ok, offs[:-1] + i + k, 0)
                ok &= (data[idx] == pat[k]) if data.size else np.zeros(n, bool)
            found |= ok
        return found
    x = c["values"].astype(np.int64)
    a = [int(v) for v in args]
    if op == "lt":
        return x < a[0]
    if op == "le":
        return x <= a[0]
    if op == "gt":
        return x > a[0]
    if op == "ge":
        return x >= a[0]
    if op == "eq":
        return x == a[0]
    if op == "ne":
        return x != a[0]
    if op == "between":
        return (x >= a[0]) & (x <= a[1])
    if op == "in":
        return np.isin(x, np.array(a, dtype=np.int64))
    raise ValueError(op)


def _probe(workload, j, fk):
    """Equi-join of the probe keys ``fk`` with join ``j``'s build side:
    (hit mask, payload arrays aligned with ``fk``).  The build side is the
    dimension's rows passing its predicates and matching every sub join of
    ``j`` (a chain), its payloads taken from its columns or from those
    sub joins' payloads."""
    dim = workload["tables"][j["dim"]]
    dc = dim["cols"]
    dm = np.ones(dim["rows"], bool)
    for p in j["preds"]:
        dm &= _pred_mask(dc, p, dim["rows"])
    sub_pay = []
    for s in j.get("joins", []):
        h, pay = _probe(workload, s, dc[s["fk"]]["values"].astype(np.int64))
        dm &= h
        sub_pay.append(pay)
    pay_cols = []
    for pc in j["payload"]:
        pay_cols.append(sub_pay[pc["join"]][pc["field"]] if isinstance(pc, dict) else dc[pc]["values"])
    keys = dc[j["key"]]["values"][dm].astype(np.int64)
    order = np.argsort(keys, kind="stable")
    skeys = keys[order]
    assert np.all(skeys[1:] != skeys[:-1]), "duplicate build keys"
    pos = np.searchsorted(skeys, fk)
    pos_c = np.minimum(pos, max(skeys.size - 1, 0))
    hit = (skeys[pos_c] == fk) if skeys.size else np.zeros(fk.size, bool)
    pay = [np.asarray(v)[dm][order][pos_c] if skeys.size else np.zeros(fk.size, np.int32) for v in pay_cols]
    return hit, pay


def evaluate(workload):
    q = workload["query"]
    fact = workload["tables"][workload["fact"]]
    n = fact["rows"]
    fc = fact["cols"]
    mask = np.ones(n, bool)
    for p in q["preds"]:
        mask &= _pred_mask(fc, p, n)
    payloads = []
    for j in q["joins"]:
        hit, pay = _probe(workload, j, fc[j["fk"]]["values"].astype(np.int64))
        mask &= hit
        payloads.append(pay)
    sel = np.nonzero(mask)[0]
    kcols = []
    for g in q["group"]:
        if "col" in g:
            kcols.append(fc[g["col"]]["values"][sel].astype(np.int64))
        else:
            kcols.append(payloads[g["join"]][g["field"]][sel].astype(np.int64))
    while len(kcols) < 2:
        kcols.append(np.zeros(sel.size, np.int64))
    if sel.size:
        stacked = np.stack(kcols, axis=1)
        uniq, inv = np.unique(stacked, axis=0, return_inverse=True)
        inv = inv.reshape(-1)
    else:
        uniq = np.zeros((0, 2), np.int64)
        inv = np.zeros(0, np.int64)
    ng = uniq.shape[0]
    out = np.zeros(ng, RECORD_DTYPE)
    out["key"] = uniq.astype(np.int32)
    out["count"] = np.bincount(inv, minlength=ng).astype(np.int64)
    for i, a in enumerate(q["aggs"]):
        if a["op"] == "count":
            out["val"][:, i] = out["count"]
            continue
        x = fc[a["cols"][0]]["values"][sel].astype(np.int64)
        if a["op"] == "sum":
            v = x
        else:
            y = fc[a["cols"][1]]["values"][sel].astype(np.int64)
            v = x * y if a["op"] == "sum_mul" else x - y
        acc = np.zeros(ng, np.int64)
        np.add.at(acc, inv, v)
        out["val"][:, i] = acc
    if not q["group"] and ng == 0:
        out = np.zeros(1, RECORD_DTYPE)
    return out
