"""Python face of the reference oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It never imports the CUDA library's
package, and the CUDA library never imports it.

``build()`` compiles ``dpf_oracle.cpp`` with the host C++ compiler into
``oracle/_build/``; everything else marshals numpy arrays through ctypes.
The arithmetic lives in the C++ file: the plain definition of the query
result (Sec. 3.1, Kernels #1-#3) evaluated row at a time, and encoders and
decoders written from the page-format definition (Sec. 3.4.1, 3.4.2, 4.1,
4.2).  See the header of ``dpf_oracle.cpp`` for what pins each part.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dpf_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

CODECS = {"for": 1, "delta": 2, "dict": 3, "str": 4, "fsst": 5, "for64": 6}
STRING_CODECS = ("str", "fsst")
PRED_OPS = {"lt": 0, "le": 1, "gt": 2, "ge": 3, "eq": 4, "ne": 5, "between": 6, "in": 7,
            "prefix": 8, "contains": 9, "like": 10}
AGG_OPS = {"count": 0, "sum": 1, "sum_mul": 2, "sum_sub": 3}

RECORD_DTYPE = np.dtype([("key", np.int32, (2,)), ("count", np.int64), ("val", np.int64, (4,))])


def build(force=False):
    """Compile the oracle library (host compiler, plain -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Column(C.Structure):
    _fields_ = [("is_str", C.c_int32), ("v", C.c_void_p), ("bytes", C.c_void_p),
                ("offsets", C.c_void_p), ("v64", C.c_void_p)]


class _Table(C.Structure):
    _fields_ = [("n", C.c_uint64), ("ncols", C.c_int32), ("cols", C.POINTER(_Column))]


class _Pred(C.Structure):
    _fields_ = [("col", C.c_int32), ("op", C.c_int32), ("nargs", C.c_int32),
                ("pfx_len", C.c_int32), ("args", C.c_int64 * 16), ("pfx", C.c_void_p)]


class _Join(C.Structure):
    pass


_Join._fields_ = [("fk_col", C.c_int32), ("dim", C.POINTER(_Table)), ("key_col", C.c_int32),
                  ("npreds", C.c_int32), ("preds", C.POINTER(_Pred)), ("npay", C.c_int32),
                  ("pay_cols", C.c_int32 * 2), ("pay_join", C.c_int32 * 2),
                  ("pay_field", C.c_int32 * 2), ("nsub", C.c_int32), ("sub", C.POINTER(_Join))]


class _Key(C.Structure):
    _fields_ = [("kind", C.c_int32), ("col", C.c_int32), ("join", C.c_int32),
                ("field", C.c_int32)]


class _Agg(C.Structure):
    _fields_ = [("op", C.c_int32), ("a", C.c_int32), ("b", C.c_int32)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            L.orc_encode_int.restype = C.c_int64
            L.orc_encode_int.argtypes = [C.c_uint32, P, C.c_uint64, C.c_uint32, P, C.c_uint64,
                                         P, P, P, C.c_uint64, P]
            L.orc_decode_int.restype = C.c_int64
            L.orc_decode_int.argtypes = [C.c_uint32, P, P, C.c_uint64, C.c_uint64, C.c_uint32,
                                         P, C.c_uint64, P]
            L.orc_decode_int_row.restype = C.c_int64
            L.orc_decode_int_row.argtypes = [C.c_uint32, P, P, P, C.c_uint64, P, C.c_uint64,
                                             C.c_uint64, P]
            L.orc_encode_for64.restype = C.c_int64
            L.orc_encode_for64.argtypes = [P, C.c_uint64, C.c_uint32, P, C.c_uint64, P, P]
            L.orc_decode_for64.restype = C.c_int64
            L.orc_decode_for64.argtypes = [P, P, C.c_uint64, C.c_uint64, C.c_uint32, P]
            L.orc_decode_for64_row.restype = C.c_int64
            L.orc_decode_for64_row.argtypes = [P, P, P, C.c_uint64, C.c_uint64, P]
            L.orc_encode_str.restype = C.c_int64
            L.orc_encode_str.argtypes = [P, P, C.c_uint64, C.c_uint32, P, C.c_uint64, P, P]
            L.orc_decode_str.restype = C.c_int64
            L.orc_decode_str.argtypes = [P, P, C.c_uint64, C.c_uint64, C.c_uint32, P, P,
                                         C.c_uint64]
            L.orc_fsst_build.restype = C.c_int64
            L.orc_fsst_build.argtypes = [P, P, C.c_uint64, P]
            L.orc_encode_fsst.restype = C.c_int64
            L.orc_encode_fsst.argtypes = [P, P, C.c_uint64, P, C.c_uint64, C.c_uint32, P, C.c_uint64, P, P]
            L.orc_decode_fsst.restype = C.c_int64
            L.orc_decode_fsst.argtypes = [P, P, C.c_uint64, C.c_uint64, C.c_uint32, P, C.c_uint64, P, P,
                                          C.c_uint64]
            L.orc_query.restype = C.c_int64
            L.orc_query.argtypes = [C.POINTER(_Table), C.c_int32, C.POINTER(_Pred), C.c_int32,
                                    C.POINTER(_Join), C.c_int32, C.POINTER(_Key), C.c_int32,
                                    C.POINTER(_Agg), P, C.c_uint64]
            L.orc_query_threads.restype = C.c_int64
            L.orc_query_threads.argtypes = L.orc_query.argtypes + [C.c_int32, C.c_uint64]
            _lib = L
    return _lib


class use_library:
    """Context manager that routes every call to another build of the
    oracle (used by the tests that plant a mistake in a copy of it)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        self._saved = lib()
        L = C.CDLL(self.path)
        for name in ("orc_encode_int", "orc_decode_int", "orc_decode_int_row", "orc_encode_for64",
                     "orc_decode_for64", "orc_decode_for64_row", "orc_encode_str", "orc_decode_str",
                     "orc_fsst_build", "orc_encode_fsst", "orc_decode_fsst", "orc_query",
                     "orc_query_threads"):
            f, g = getattr(L, name), getattr(self._saved, name)
            f.restype, f.argtypes = g.restype, g.argtypes
        _lib = L
        return L

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def _ptr(a):
    return a.ctypes.data if a is not None and a.size else None


class OracleError(RuntimeError):
    pass


def _check(rc, what):
    if rc < 0:
        raise OracleError(f"{what} failed with status {rc}")
    return rc


# ---------------------------------------------------------------------------
# Encoding / decoding
# ---------------------------------------------------------------------------

def encode_column(col, page_rows):
    """Encode one column dict (see ``synth``) into the page format.

    Returns ``{"codec", "rows", "page_rows", "blob", "page_off", "row_prefix",
    "dict"}`` with numpy arrays.
    """
    L = lib()
    codec = col["codec"]
    if codec == "fsst":
        offsets = np.ascontiguousarray(col["offsets"], dtype=np.uint64)
        data = np.ascontiguousarray(col["bytes"], dtype=np.uint8)
        n = offsets.size - 1
        table = col.get("table")
        if table is None:
            table = np.zeros(3 * 255, np.int32)
            nsym = _check(L.orc_fsst_build(_ptr(data) or offsets.ctypes.data, _ptr(offsets), n,
                                           _ptr(table)), "fsst_build")
            table = table[: 3 * nsym].copy()
        table = np.ascontiguousarray(table, np.int32)
        npages = (n + page_rows - 1) // page_rows
        page_off = np.zeros(npages + 1, np.uint64)
        row_prefix = np.zeros(npages, np.uint64)
        args = (_ptr(data) or offsets.ctypes.data, _ptr(offsets), n, _ptr(table) or offsets.ctypes.data,
                table.size, page_rows)
        size = _check(L.orc_encode_fsst(*args, None, 0, _ptr(page_off), _ptr(row_prefix)), "encode_fsst")
        blob = np.zeros(size, np.uint8)
        _check(L.orc_encode_fsst(*args, _ptr(blob), size, _ptr(page_off), _ptr(row_prefix)), "encode_fsst")
        return {"codec": codec, "rows": n, "page_rows": page_rows, "blob": blob,
                "page_off": page_off, "row_prefix": row_prefix, "dict": table}
    if codec == "str":
        offsets = np.ascontiguousarray(col["offsets"], dtype=np.uint64)
        data = np.ascontiguousarray(col["bytes"], dtype=np.uint8)
        n = offsets.size - 1
        npages = (n + page_rows - 1) // page_rows
        page_off = np.zeros(npages + 1, np.uint64)
        row_prefix = np.zeros(npages, np.uint64)
        size = _check(L.orc_encode_str(_ptr(data), _ptr(offsets), n, page_rows, None, 0,
                                       _ptr(page_off), _ptr(row_prefix)), "encode_str")
        blob = np.zeros(size, np.uint8)
        _check(L.orc_encode_str(_ptr(data), _ptr(offsets), n, page_rows, _ptr(blob), size,
                                _ptr(page_off), _ptr(row_prefix)), "encode_str")
        return {"codec": codec, "rows": n, "page_rows": page_rows, "blob": blob,
                "page_off": page_off, "row_prefix": row_prefix, "dict": None}
    if codec == "for64":
        v = np.ascontiguousarray(col["values"], dtype=np.int64)
        n = v.size
        npages = (n + page_rows - 1) // page_rows
        page_off = np.zeros(npages + 1, np.uint64)
        row_prefix = np.zeros(npages, np.uint64)
        size = _check(L.orc_encode_for64(_ptr(v), n, page_rows, None, 0, _ptr(page_off), _ptr(row_prefix)),
                      "encode_for64")
        blob = np.zeros(size, np.uint8)
        _check(L.orc_encode_for64(_ptr(v), n, page_rows, _ptr(blob), size, _ptr(page_off), _ptr(row_prefix)),
               "encode_for64")
        return {"codec": codec, "rows": n, "page_rows": page_rows, "blob": blob,
                "page_off": page_off, "row_prefix": row_prefix, "dict": None}
    v = np.ascontiguousarray(col["values"], dtype=np.int32)
    n = v.size
    npages = (n + page_rows - 1) // page_rows
    page_off = np.zeros(npages + 1, np.uint64)
    row_prefix = np.zeros(npages, np.uint64)
    dict_n = np.zeros(1, np.uint64)
    size = _check(L.orc_encode_int(CODECS[codec], _ptr(v), n, page_rows, None, 0,
                                   _ptr(page_off), _ptr(row_prefix), None, 0, _ptr(dict_n)),
                  "encode_int")
    blob = np.zeros(size, np.uint8)
    dct = np.zeros(max(int(dict_n[0]), 1), np.int32) if codec == "dict" else None
    _check(L.orc_encode_int(CODECS[codec], _ptr(v), n, page_rows, _ptr(blob), size,
                            _ptr(page_off), _ptr(row_prefix), _ptr(dct),
                            0 if dct is None else dct.size, _ptr(dict_n)), "encode_int")
    if dct is not None:
        dct = dct[: int(dict_n[0])]
    return {"codec": codec, "rows": n, "page_rows": page_rows, "blob": blob,
            "page_off": page_off, "row_prefix": row_prefix, "dict": dct}


def _decode_pages_threaded(enc, threads):
    """Integer columns: the pages cut into ``threads`` contiguous ranges, each
    decoded by the same C decoder on its own host thread (ctypes releases the
    interpreter lock during the call) into its slice of the output."""
    import concurrent.futures as cf
    L = lib()
    n, npages, P = enc["rows"], enc["page_off"].size - 1, enc["page_rows"]
    wide = enc["codec"] == "for64"
    out = np.zeros(n, np.int64 if wide else np.int32)
    item = out.itemsize
    dct = enc["dict"]
    bounds = np.linspace(0, npages, min(threads, npages) + 1).astype(np.int64)
    po = enc["page_off"].ctypes.data

    def work(k):
        p0, p1 = int(bounds[k]), int(bounds[k + 1])
        if p1 <= p0:
            return 0
        rows = min(n, p1 * P) - p0 * P
        dst = out.ctypes.data + item * p0 * P
        if wide:
            return L.orc_decode_for64(_ptr(enc["blob"]), po + 8 * p0, p1 - p0, rows, P, dst)
        return L.orc_decode_int(CODECS[enc["codec"]], _ptr(enc["blob"]), po + 8 * p0, p1 - p0, rows, P,
                                _ptr(dct), 0 if dct is None else dct.size, dst)

    with cf.ThreadPoolExecutor(max_workers=len(bounds) - 1) as ex:
        for rc in ex.map(work, range(len(bounds) - 1)):
            _check(rc, "decode (threaded)")
    return out


def decode_column(enc, threads=1):
    """Decode a whole encoded column: int32 values, or (bytes, offsets).
    ``threads`` > 1 decodes integer columns page range by page range on
    that many host threads (the same decoder; the rows are identical)."""
    L = lib()
    n, npages = enc["rows"], enc["page_off"].size - 1
    if threads > 1 and npages > 1 and enc["codec"] in ("for", "delta", "dict", "for64"):
        return _decode_pages_threaded(enc, threads)
    if enc["codec"] == "fsst":
        offsets = np.zeros(n + 1, np.uint64)
        table = np.ascontiguousarray(enc["dict"], np.int32)
        cap = 8 * max(enc["blob"].size, 1)  # a code expands to at most 8 bytes
        data = np.zeros(cap, np.uint8)
        _check(L.orc_decode_fsst(_ptr(enc["blob"]), _ptr(enc["page_off"]), npages, n, enc["page_rows"],
                                 _ptr(table) or offsets.ctypes.data, table.size, _ptr(offsets), _ptr(data),
                                 data.size), "decode_fsst")
        return data[: int(offsets[-1])].copy(), offsets
    if enc["codec"] == "str":
        # byte count = blob bytes is an upper bound on the string bytes
        offsets = np.zeros(n + 1, np.uint64)
        data = np.zeros(max(enc["blob"].size, 1), np.uint8)
        _check(L.orc_decode_str(_ptr(enc["blob"]), _ptr(enc["page_off"]), npages, n,
                                enc["page_rows"], _ptr(offsets), _ptr(data), data.size),
               "decode_str")
        return data[: int(offsets[-1])].copy(), offsets
    if enc["codec"] == "for64":
        out = np.zeros(n, np.int64)
        _check(L.orc_decode_for64(_ptr(enc["blob"]), _ptr(enc["page_off"]), npages, n, enc["page_rows"],
                                  _ptr(out)), "decode_for64")
        return out
    out = np.zeros(n, np.int32)
    dct = enc["dict"]
    _check(L.orc_decode_int(CODECS[enc["codec"]], _ptr(enc["blob"]), _ptr(enc["page_off"]),
                            npages, n, enc["page_rows"], _ptr(dct),
                            0 if dct is None else dct.size, _ptr(out)), "decode_int")
    return out


def decode_row(enc, r):
    """Decode the single value at row ``r`` through the RID index."""
    L = lib()
    if enc["codec"] == "for64":
        out = np.zeros(1, np.int64)
        _check(L.orc_decode_for64_row(_ptr(enc["blob"]), _ptr(enc["page_off"]), _ptr(enc["row_prefix"]),
                                      enc["page_off"].size - 1, int(r), _ptr(out)), "decode_for64_row")
        return int(out[0])
    out = np.zeros(1, np.int32)
    dct = enc["dict"]
    _check(L.orc_decode_int_row(CODECS[enc["codec"]], _ptr(enc["blob"]), _ptr(enc["page_off"]),
                                _ptr(enc["row_prefix"]), enc["page_off"].size - 1, _ptr(dct),
                                0 if dct is None else dct.size, int(r), _ptr(out)),
           "decode_int_row")
    return int(out[0])


# ---------------------------------------------------------------------------
# Query evaluation
# ---------------------------------------------------------------------------

def _make_pred(pred, names):
    p = _Pred()
    p.col = names.index(pred["col"])
    p.op = PRED_OPS[pred["op"]]
    if pred["op"] in ("prefix", "contains", "like"):
        pfx = bytes(pred["args"][0])
        buf = C.create_string_buffer(pfx, max(len(pfx), 1))
        p.pfx = C.cast(buf, C.c_void_p)
        p.pfx_len = len(pfx)
        p.nargs = 0
        return p, buf
    args = [int(a) for a in pred["args"]]
    if len(args) > 16:
        raise ValueError("at most 16 predicate operands")
    p.nargs = len(args)
    for i, a in enumerate(args):
        p.args[i] = a
    return p, None


def _table(cols, n):
    names = list(cols)
    arr = (_Column * max(len(names), 1))()
    keep = []
    for i, name in enumerate(names):
        c = cols[name]
        if isinstance(c, tuple):
            data, offs = c
            data = np.ascontiguousarray(data, np.uint8)
            offs = np.ascontiguousarray(offs, np.uint64)
            keep += [data, offs]
            arr[i].is_str = 1
            arr[i].bytes = _ptr(data) if data.size else offs.ctypes.data  # never read when empty
            arr[i].offsets = _ptr(offs)
        elif np.asarray(c).dtype == np.int64:  # a 64-bit (FOR64) column
            v = np.ascontiguousarray(c, np.int64)
            keep.append(v)
            arr[i].is_str = 0
            arr[i].v64 = _ptr(v)
        else:
            v = np.ascontiguousarray(c, np.int32)
            keep.append(v)
            arr[i].is_str = 0
            arr[i].v = _ptr(v)
    t = _Table(n, len(names), C.cast(arr, C.POINTER(_Column)))
    keep.append(arr)
    return t, names, keep


def decoded_tables(workload, from_encoded=True, threads=1, encoded=None):
    """Every table's columns, decoded through the oracle's own encoder and
    decoder (``from_encoded``) or taken raw from the generator.  ``encoded``
    maps (table, column) to pages already encoded by ``encode_tables``."""
    out = {}
    for tname, t in workload["tables"].items():
        cols = {}
        for cname, c in t["cols"].items():
            if from_encoded:
                enc = encoded[(tname, cname)] if encoded else encode_column(c, t["page_rows"])
                d = decode_column(enc, threads)
                cols[cname] = d
            else:
                cols[cname] = (c["bytes"], c["offsets"]) if c["codec"] in STRING_CODECS else c["values"]
        out[tname] = {"rows": t["rows"], "cols": cols}
    return out


def encode_tables(workload):
    """Every column of every table through the oracle's encoder (the loader:
    a step that precedes the query and is timed apart from it)."""
    return {(tname, cname): encode_column(c, t["page_rows"])
            for tname, t in workload["tables"].items() for cname, c in t["cols"].items()}


def _joins(tables, specs, probe_names, keep, dim_tables):
    """ctypes array of the joins ``specs`` probed from a table with columns
    ``probe_names``; a join's own ``joins`` (a chain) are probed from its
    dimension and become its sub joins."""
    arr = (_Join * max(len(specs), 1))()
    for i, j in enumerate(specs):
        d = tables[j["dim"]]
        dt, dnames, dkeep = _table(d["cols"], d["rows"])
        keep += dkeep
        dim_tables.append(dt)
        dp = (_Pred * max(len(j["preds"]), 1))()
        for k, pr in enumerate(j["preds"]):
            dp[k], buf = _make_pred(pr, dnames)
            keep.append(buf)
        keep.append(dp)
        subs = j.get("joins", [])
        sub = _joins(tables, subs, dnames, keep, dim_tables)
        arr[i].fk_col = probe_names.index(j["fk"])
        arr[i].dim = C.pointer(dt)
        arr[i].key_col = dnames.index(j["key"])
        arr[i].npreds = len(j["preds"])
        arr[i].preds = C.cast(dp, C.POINTER(_Pred))
        arr[i].npay = len(j["payload"])
        for f, pc in enumerate(j["payload"]):
            if isinstance(pc, dict):
                arr[i].pay_cols[f], arr[i].pay_join[f], arr[i].pay_field[f] = 0, pc["join"], pc["field"]
            else:
                arr[i].pay_cols[f], arr[i].pay_join[f], arr[i].pay_field[f] = dnames.index(pc), -1, 0
        arr[i].nsub = len(subs)
        arr[i].sub = C.cast(sub, C.POINTER(_Join))
    keep.append(arr)
    return arr


def host_threads():
    """Host threads the oracle may use: the CPUs this process may run on."""
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except (AttributeError, OSError):
        return max(1, os.cpu_count() or 1)


def run_query(workload, from_encoded=True, tables=None, threads=1, encoded=None):
    """Evaluate ``workload['query']``; returns an array of RECORD_DTYPE.

    ``threads`` > 1 evaluates the fact table's pages on that many host
    threads (``orc_query_threads``: disjoint page ranges, per-thread group
    maps added together); ``threads=0`` uses every CPU of the process."""
    L = lib()
    if threads == 0:
        threads = host_threads()
    if tables is None and encoded is not None:
        tables = decoded_tables(workload, True, threads, encoded)
    q = workload["query"]
    if tables is None:
        tables = decoded_tables(workload, from_encoded, threads)
    fact = tables[workload["fact"]]
    ft, fnames, keep = _table(fact["cols"], fact["rows"])
    preds = (_Pred * max(len(q["preds"]), 1))()
    for i, pr in enumerate(q["preds"]):
        preds[i], buf = _make_pred(pr, fnames)
        keep.append(buf)
    dim_tables = []
    joins = _joins(tables, q["joins"], fnames, keep, dim_tables)
    keys = (_Key * max(len(q["group"]), 1))()
    for i, g in enumerate(q["group"]):
        if "col" in g:
            keys[i].kind, keys[i].col = 0, fnames.index(g["col"])
        else:
            keys[i].kind, keys[i].join, keys[i].field = 1, g["join"], g["field"]
    aggs = (_Agg * max(len(q["aggs"]), 1))()
    for i, a in enumerate(q["aggs"]):
        aggs[i].op = AGG_OPS[a["op"]]
        cols = a.get("cols", [])
        aggs[i].a = fnames.index(cols[0]) if cols else 0
        aggs[i].b = fnames.index(cols[1]) if len(cols) > 1 else 0
    page_rows = int(workload["tables"][workload["fact"]].get("page_rows", 65536))

    def call(out, cap):
        args = (C.pointer(ft), len(q["preds"]), preds, len(q["joins"]), joins,
                len(q["group"]), keys, len(q["aggs"]), aggs, _ptr(out), cap)
        if threads > 1:
            return _check(L.orc_query_threads(*args, int(threads), page_rows), "query_threads")
        return _check(L.orc_query(*args), "query")

    cap = 1 << 16
    out = np.zeros(cap, RECORD_DTYPE)
    n = call(out, cap)
    if n > cap:
        out = np.zeros(n, RECORD_DTYPE)
        n = call(out, n)
    del keep, dim_tables
    return out[:n].copy()
