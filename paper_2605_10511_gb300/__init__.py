"""Python binding of the fused columnar query library (``include/dpf.h``).

Argument marshalling only: every step of the query path runs in the CUDA
library ``_build/libdpf.so`` (built by ``_build.build()``).  If the library
cannot be built or loaded, every call raises ``DpfUnavailable``; there is no
CPU fallback.

PyTorch supplies device memory (through the allocation hooks, when
``use_torch_allocator`` is set) and streams (``torch.cuda.current_stream``).
"""

from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

DPF_OK = 0
STATUS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "EDUPKEY", -5: "EBUSY", -6: "ETIMEOUT",
          -7: "ETRUNC", -8: "ENOTFOUND", -9: "ECORRUPT", -10: "EINTERNAL"}
CODEC = {"for": 1, "delta": 2, "dict": 3, "str": 4, "fsst": 5, "for64": 6}
STRING_CODECS = ("str", "fsst")
PLACE = {"device": 0, "host": 1}
OP = {"lt": 0, "le": 1, "gt": 2, "ge": 3, "eq": 4, "ne": 5, "between": 6, "in": 7, "prefix": 8,
      "contains": 9, "like": 10}
AGG = {"count": 0, "sum": 1, "sum_mul": 2, "sum_sub": 3}
HT_PLACE = {"auto": 0, "smem": 1, "global": 2}
MAX_IN = 8
MAX_PREFIX = 32

RECORD_DTYPE = np.dtype([("key", np.int32, (2,)), ("count", np.int64), ("val", np.int64, (4,))])


class DpfUnavailable(RuntimeError):
    """The CUDA library is not built or cannot be loaded."""


class DpfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class ColumnDesc(C.Structure):
    _fields_ = [("codec", C.c_int32), ("placement", C.c_int32), ("page_rows", C.c_uint32),
                ("table", C.c_int32)]


class Pred(C.Structure):
    _fields_ = [("col", C.c_int32), ("op", C.c_int32), ("n", C.c_int32), ("prefix_len", C.c_int32),
                ("v", C.c_int64 * MAX_IN), ("prefix", C.c_uint8 * MAX_PREFIX)]


class Join(C.Structure):
    _fields_ = [("fk_col", C.c_int32), ("ht", C.c_int32)]


class Payload(C.Structure):
    _fields_ = [("kind", C.c_int32), ("col", C.c_int32), ("join", C.c_int32), ("field", C.c_int32)]


class Build(C.Structure):
    _fields_ = [("key_col", C.c_int32), ("n_payload", C.c_int32), ("payload", C.POINTER(Payload)),
                ("n_preds", C.c_int32), ("preds", C.POINTER(Pred)),
                ("n_joins", C.c_int32), ("joins", C.POINTER(Join))]


class Key(C.Structure):
    _fields_ = [("kind", C.c_int32), ("col", C.c_int32), ("join", C.c_int32), ("field", C.c_int32)]


class Agg(C.Structure):
    _fields_ = [("op", C.c_int32), ("a", C.c_int32), ("b", C.c_int32)]


class Plan(C.Structure):
    _fields_ = [("n_preds", C.c_int32), ("preds", C.POINTER(Pred)),
                ("n_joins", C.c_int32), ("joins", C.POINTER(Join)),
                ("n_keys", C.c_int32), ("keys", C.POINTER(Key)),
                ("n_aggs", C.c_int32), ("aggs", C.POINTER(Agg)), ("scan_col", C.c_int32)]


class Tuning(C.Structure):
    _fields_ = [("chunk_rows", C.c_uint32), ("threads", C.c_uint32), ("ht_placement", C.c_int32),
                ("ctas_per_sm", C.c_uint32), ("staging", C.c_int32), ("group_agg", C.c_int32)]


STAGING = {"default": 0, "on": 1, "off": 2}
GROUP_AGG = {"default": 0, "warp": 1, "atomic": 2}


class ServerConfig(C.Structure):
    _fields_ = [("max_batch", C.c_uint32), ("max_inflight", C.c_uint32), ("mem_budget", C.c_uint64),
                ("tuning", Tuning)]


class QueryTimes(C.Structure):
    _fields_ = [("submit_us", C.c_double), ("launch_us", C.c_double), ("done_us", C.c_double),
                ("batch_size", C.c_uint32)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("batches", C.c_uint64), ("launched_batches", C.c_uint64), ("queued", C.c_uint64),
                ("in_use_bytes", C.c_uint64)]


class AllocHooks(C.Structure):
    _fields_ = [("alloc", C.CFUNCTYPE(C.c_void_p, C.c_uint64, C.c_void_p)),
                ("free", C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)),
                ("user", C.c_void_p)]


# every symbol of include/dpf.h with its ctypes signature
_P = C.c_void_p
_SIGS = {
    "dpf_last_error": (C.c_char_p, []),
    "dpf_create": (C.c_int32, [C.POINTER(_P), C.c_int32, C.c_uint64, C.POINTER(AllocHooks)]),
    "dpf_destroy": (C.c_int32, [_P]),
    "dpf_memory_used": (C.c_int32, [_P, C.POINTER(C.c_uint64)]),
    "dpf_context_device": (C.c_int32, [_P, C.POINTER(C.c_int32)]),
    "dpf_encode_column": (C.c_int32, [C.POINTER(ColumnDesc), _P, _P, C.c_uint64, _P, C.c_uint64, _P, _P,
                                      _P, C.c_uint64, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
    "dpf_load_encoded": (C.c_int32, [_P, C.POINTER(ColumnDesc), _P, C.c_uint64, _P, _P, C.c_uint64, _P,
                                     C.c_uint64, C.POINTER(C.c_int32)]),
    "dpf_load_column": (C.c_int32, [_P, C.POINTER(ColumnDesc), _P, _P, C.c_uint64, C.POINTER(C.c_int32)]),
    "dpf_column_info": (C.c_int32, [_P, C.c_int32, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64),
                                    C.POINTER(C.c_uint64)]),
    "dpf_column_read": (C.c_int32, [_P, C.c_int32, C.c_uint64, C.c_uint64, _P]),
    "dpf_drop_column": (C.c_int32, [_P, C.c_int32]),
    "dpf_build_hash": (C.c_int32, [_P, C.c_int32, _P, C.c_int32, C.POINTER(Pred), C.c_int32, _P,
                                   C.POINTER(C.c_int32)]),
    "dpf_build_hash_probe": (C.c_int32, [_P, C.POINTER(Build), _P, C.POINTER(C.c_int32)]),
    "dpf_build_hash_async": (C.c_int32, [_P, C.POINTER(Build), _P, C.POINTER(C.c_int32)]),
    "dpf_hash_wait": (C.c_int32, [_P, C.c_int32]),
    "dpf_set_tuning": (C.c_int32, [_P, C.c_char_p]),
    "dpf_parse_tuning": (C.c_int32, [C.c_char_p, C.POINTER(Tuning)]),
    "dpf_build_hash_deferred": (C.c_int32, [_P, C.POINTER(Build), C.POINTER(C.c_int32)]),
    "dpf_prepare_chain": (C.c_int32, [_P, C.POINTER(C.c_int32), C.c_int32, C.POINTER(Plan), C.c_int32,
                                      C.POINTER(Tuning), C.POINTER(C.c_int32)]),
    "dpf_hash_info": (C.c_int32, [_P, C.c_int32, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
    "dpf_drop_hash": (C.c_int32, [_P, C.c_int32]),
    "dpf_prepare": (C.c_int32, [_P, C.POINTER(Plan), C.c_int32, C.POINTER(Tuning), C.POINTER(C.c_int32)]),
    "dpf_launch": (C.c_int32, [_P, C.c_int32, _P]),
    "dpf_capture_graph": (C.c_int32, [_P, C.c_int32, _P]),
    "dpf_launch_graph": (C.c_int32, [_P, C.c_int32, _P]),
    "dpf_read_result": (C.c_int32, [_P, C.c_int32, C.c_int32, _P, C.c_uint64, C.POINTER(C.c_uint64),
                                    C.c_int32]),
    "dpf_prep_tuning": (C.c_int32, [_P, C.c_int32, C.POINTER(Tuning)]),
    "dpf_release": (C.c_int32, [_P, C.c_int32]),
    "dpf_autotune": (C.c_int32, [_P, C.POINTER(Plan), C.c_int32, _P, C.c_uint32, C.POINTER(Tuning),
                                 C.POINTER(C.c_float)]),
    "dpf_plan_footprint": (C.c_int32, [_P, C.POINTER(Plan), C.POINTER(C.c_uint64)]),
    "dpf_prepare_unfused": (C.c_int32, [_P, C.POINTER(Plan), C.POINTER(C.c_int32)]),
    "dpf_prep_stats": (C.c_int32, [_P, C.c_int32, C.POINTER(C.c_uint32), C.POINTER(C.c_uint64)]),
    "dpf_execute_noalloc": (C.c_int32, [_P, C.POINTER(Plan), _P, _P, C.c_uint64, _P]),
    "dpf_noalloc_status": (C.c_int32, [_P, C.POINTER(C.c_uint32)]),
    "dpf_read_rate": (C.c_int32, [_P, C.c_int32, C.c_uint64, C.c_uint32, _P, C.POINTER(C.c_double)]),
    "dpf_execute_plan": (C.c_int32, [_P, C.POINTER(Plan), C.c_int32, _P, C.POINTER(C.c_int64)]),
    "dpf_fetch_result": (C.c_int32, [_P, C.c_int64, _P, C.c_uint64, C.POINTER(C.c_uint64), C.c_int32]),
    "dpf_server_create": (C.c_int32, [_P, C.POINTER(ServerConfig), C.POINTER(_P)]),
    "dpf_server_submit": (C.c_int32, [_P, C.POINTER(Plan), C.POINTER(C.c_uint64)]),
    "dpf_server_wait": (C.c_int32, [_P, C.c_uint64, _P, C.c_uint64, C.POINTER(C.c_uint64), C.c_int32,
                                    C.POINTER(QueryTimes)]),
    "dpf_server_stats_get": (C.c_int32, [_P, C.POINTER(ServerStats)]),
    "dpf_server_destroy": (C.c_int32, [_P]),
}

_lock = threading.Lock()
_lib = None


def library_path():
    return _build.LIB


def build(force=False):
    """Compile the CUDA library for sm_103a (nvcc)."""
    return _build.build(force=force)


def lib():
    """The loaded library; builds it first if it is missing or stale."""
    global _lib
    with _lock:
        if _lib is None:
            try:
                path = _build.build()
            except Exception as exc:  # noqa: BLE001
                raise DpfUnavailable(f"cannot build the CUDA library: {exc}") from exc
            try:
                L = C.CDLL(path)
            except OSError as exc:
                raise DpfUnavailable(f"cannot load {path}: {exc}") from exc
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(st):
    if st != DPF_OK:
        msg = lib().dpf_last_error()
        raise DpfError(st, msg.decode() if msg else "")


def _ptr(a):
    return C.c_void_p(a.ctypes.data) if a is not None else None


def _stream_ptr(stream):
    """cudaStream_t of a torch stream (or an int handle, or None = current)."""
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def parse_tuning(text):
    """The launch configuration a JSON object string gives (``dpf_parse_tuning``,
    host only): a dict of the dpf_tuning fields."""
    t = Tuning()
    _check(lib().dpf_parse_tuning(None if text is None else text.encode(), C.byref(t)))
    return {f: getattr(t, f) for f, _ in Tuning._fields_}


def make_pred(col_id, op, args):
    p = Pred()
    p.col = col_id
    p.op = OP[op]
    if op in ("prefix", "contains", "like"):
        pfx = bytes(args[0])
        if len(pfx) > MAX_PREFIX:
            raise ValueError(f"pattern longer than {MAX_PREFIX} bytes")
        p.prefix_len = len(pfx)
        for i, b in enumerate(pfx):
            p.prefix[i] = b
        return p
    vals = [int(a) for a in args]
    if len(vals) > MAX_IN:
        raise ValueError(f"at most {MAX_IN} operands")
    p.n = len(vals)
    for i, v in enumerate(vals):
        p.v[i] = v
    return p


class Context:
    """One library context on one CUDA device."""

    def __init__(self, device=0, hbm_budget=0, use_torch_allocator=False):
        L = lib()
        self._hooks = None
        hooks_ptr = None
        if use_torch_allocator:
            import torch
            dev = int(device)

            @C.CFUNCTYPE(C.c_void_p, C.c_uint64, C.c_void_p)
            def _alloc(n, _user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(n), device=dev)
                except Exception:  # noqa: BLE001 - reported to the library as NULL
                    return None

            @C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)
            def _free(p, _user):
                torch.cuda.caching_allocator_delete(p)

            self._hooks = AllocHooks(_alloc, _free, None)
            hooks_ptr = C.pointer(self._hooks)
        h = C.c_void_p()
        _check(L.dpf_create(C.byref(h), int(device), int(hbm_budget), hooks_ptr))
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            lib().dpf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    # ------------------------------------------------------------ columns
    def load_column(self, col, table=0, page_rows=0, placement="device"):
        """Load one column dict (``{"codec", "values"}``, int64 values for
        ``for64``, or ``{"codec": "str" or "fsst", "bytes", "offsets"}``);
        returns its id."""
        d = ColumnDesc(CODEC[col["codec"]], PLACE[placement], int(page_rows), int(table))
        out = C.c_int32()
        if col["codec"] in STRING_CODECS:
            data = np.ascontiguousarray(col["bytes"], np.uint8)
            offs = np.ascontiguousarray(col["offsets"], np.uint64)
            src = data if data.size else np.zeros(1, np.uint8)
            _check(lib().dpf_load_column(self.h, C.byref(d), _ptr(src), _ptr(offs), offs.size - 1,
                                         C.byref(out)))
        else:
            v = np.ascontiguousarray(col["values"], np.int64 if col["codec"] == "for64" else np.int32)
            _check(lib().dpf_load_column(self.h, C.byref(d), _ptr(v), None, v.size, C.byref(out)))
        return out.value

    def load_encoded(self, enc, table=0, placement="device"):
        """Upload pages produced by ``encode_column``."""
        d = ColumnDesc(CODEC[enc["codec"]], PLACE[placement], int(enc["page_rows"]), int(table))
        out = C.c_int32()
        dct = enc.get("dict")
        _check(lib().dpf_load_encoded(self.h, C.byref(d), _ptr(enc["blob"]), enc["blob"].size,
                                      _ptr(enc["page_off"]), _ptr(enc["row_prefix"]), enc["rows"],
                                      _ptr(dct) if dct is not None else None,
                                      0 if dct is None else dct.size, C.byref(out)))
        return out.value

    def column_info(self, cid):
        r, e, w = C.c_uint64(), C.c_uint64(), C.c_uint64()
        _check(lib().dpf_column_info(self.h, cid, C.byref(r), C.byref(e), C.byref(w)))
        return {"rows": r.value, "encoded_bytes": e.value, "raw_bytes": w.value}

    def column_bytes(self, cid):
        n = self.column_info(cid)["encoded_bytes"]
        out = np.zeros(n, np.uint8)
        _check(lib().dpf_column_read(self.h, cid, 0, n, _ptr(out)))
        return out

    def drop_column(self, cid):
        _check(lib().dpf_drop_column(self.h, cid))

    def memory_used(self):
        x = C.c_uint64()
        _check(lib().dpf_memory_used(self.h, C.byref(x)))
        return x.value

    # ------------------------------------------------------------ hash tables
    def build_hash(self, key_col, payload_cols=(), preds=(), stream=None):
        pay = np.array(list(payload_cols) or [0], np.int32)
        parr = (Pred * max(len(preds), 1))(*preds)
        out = C.c_int32()
        _check(lib().dpf_build_hash(self.h, key_col, _ptr(pay), len(payload_cols), parr, len(preds),
                                    _stream_ptr(stream), C.byref(out)))
        return out.value

    def build_hash_probe(self, key_col, payload=(), preds=(), joins=(), stream=None, asynchronous=False,
                         deferred=False):
        """Scan, probe and build (one link of a join chain).  ``payload``
        items are a DICT column id or ``("join", j, field)``: payload
        ``field`` of the row's match in ``joins[j]``; ``joins`` are
        ``(fk_col, ht)`` pairs probed from the scanned table.  With
        ``asynchronous`` the table is sized from load-time bounds and the
        call only enqueues (``dpf_build_hash_async``; ``hash_wait`` reports
        what the kernels found)."""
        pay = (Payload * max(len(payload), 1))()
        for i, p in enumerate(payload):
            pay[i] = Payload(1, 0, p[1], p[2]) if isinstance(p, tuple) else Payload(0, p, 0, 0)
        parr = (Pred * max(len(preds), 1))(*preds)
        jarr = (Join * max(len(joins), 1))(*[Join(fk, ht) for fk, ht in joins])
        b = Build(key_col, len(payload), C.cast(pay, C.POINTER(Payload)), len(preds),
                  C.cast(parr, C.POINTER(Pred)), len(joins), C.cast(jarr, C.POINTER(Join)))
        out = C.c_int32()
        if deferred:
            _check(lib().dpf_build_hash_deferred(self.h, C.byref(b), C.byref(out)))
        else:
            call = lib().dpf_build_hash_async if asynchronous else lib().dpf_build_hash_probe
            _check(call(self.h, C.byref(b), _stream_ptr(stream), C.byref(out)))
        return out.value

    def build_hash_async(self, key_col, payload=(), preds=(), joins=(), stream=None):
        return self.build_hash_probe(key_col, payload, preds, joins, stream, asynchronous=True)

    def build_hash_deferred(self, key_col, payload=(), preds=(), joins=()):
        """A table prepared but not built (``dpf_build_hash_deferred``): empty
        until a chain prepared with ``prepare_chain`` runs it."""
        return self.build_hash_probe(key_col, payload, preds, joins, deferred=True)

    def hash_wait(self, ht):
        _check(lib().dpf_hash_wait(self.h, ht))

    def hash_info(self, ht):
        e, c = C.c_uint64(), C.c_uint64()
        _check(lib().dpf_hash_info(self.h, ht, C.byref(e), C.byref(c)))
        return {"entries": e.value, "capacity": c.value}

    def drop_hash(self, ht):
        _check(lib().dpf_drop_hash(self.h, ht))

    # ------------------------------------------------------------ execution
    def prepare(self, plans, tuning=None):
        arr = (Plan * len(plans))(*[p.plan for p in plans])
        out = C.c_int32()
        _check(lib().dpf_prepare(self.h, arr, len(plans), C.byref(tuning) if tuning else None,
                                 C.byref(out)))
        return out.value

    def set_tuning(self, tuning=None):
        """The context's default launch configuration (``dpf_set_tuning``):
        a dict or a JSON object string; None resets."""
        import json
        text = None if tuning is None else (tuning if isinstance(tuning, str) else json.dumps(tuning))
        _check(lib().dpf_set_tuning(self.h, None if text is None else text.encode()))

    def prepare_chain(self, builds, plans, tuning=None):
        """A batch whose every launch rebuilds the deferred tables ``builds``
        (inner tables first) and then runs ``plans`` (``dpf_prepare_chain``)."""
        ids = (C.c_int32 * len(builds))(*builds)
        arr = (Plan * len(plans))(*[p.plan for p in plans])
        out = C.c_int32()
        _check(lib().dpf_prepare_chain(self.h, ids, len(builds), arr, len(plans),
                                       C.byref(tuning) if tuning else None, C.byref(out)))
        return out.value

    def launch(self, prep, stream=None):
        _check(lib().dpf_launch(self.h, prep, _stream_ptr(stream)))

    def capture_graph(self, prep, stream):
        _check(lib().dpf_capture_graph(self.h, prep, _stream_ptr(stream)))

    def launch_graph(self, prep, stream=None):
        _check(lib().dpf_launch_graph(self.h, prep, _stream_ptr(stream)))

    def read_result(self, prep, i=0, timeout_ms=-1):
        n = C.c_uint64()
        cap = 1024
        while True:
            buf = np.zeros(cap, RECORD_DTYPE)
            st = lib().dpf_read_result(self.h, prep, i, _ptr(buf), cap, C.byref(n), timeout_ms)
            if st == -7:
                cap = int(n.value)
                continue
            _check(st)
            return buf[: n.value].copy()

    def prep_tuning(self, prep):
        t = Tuning()
        _check(lib().dpf_prep_tuning(self.h, prep, C.byref(t)))
        return {"chunk_rows": t.chunk_rows, "threads": t.threads, "ht_placement": t.ht_placement,
                "ctas_per_sm": t.ctas_per_sm, "staging": t.staging, "group_agg": t.group_agg}

    def autotune(self, plans, stream=None, reps=3):
        """Times the plans under the library's grid of launch configurations
        and caches the fastest for them; returns (tuning dict, ms/launch)."""
        arr = (Plan * len(plans))(*[p.plan for p in plans])
        t, ms = Tuning(), C.c_float()
        _check(lib().dpf_autotune(self.h, arr, len(plans), _stream_ptr(stream), reps, C.byref(t), C.byref(ms)))
        return ({"chunk_rows": t.chunk_rows, "threads": t.threads, "ht_placement": t.ht_placement,
                 "ctas_per_sm": t.ctas_per_sm, "staging": t.staging, "group_agg": t.group_agg}, ms.value)

    def plan_footprint(self, plan):
        b = C.c_uint64()
        _check(lib().dpf_plan_footprint(self.h, C.byref(plan.plan), C.byref(b)))
        return b.value

    def device(self):
        d = C.c_int32()
        _check(lib().dpf_context_device(self.h, C.byref(d)))
        return d.value

    def prepare_unfused(self, plan):
        out = C.c_int32()
        _check(lib().dpf_prepare_unfused(self.h, C.byref(plan.plan), C.byref(out)))
        return out.value

    def prep_stats(self, prep):
        n, b = C.c_uint32(), C.c_uint64()
        _check(lib().dpf_prep_stats(self.h, prep, C.byref(n), C.byref(b)))
        return {"launches": n.value, "intermediate_bytes": b.value}

    def release(self, prep):
        _check(lib().dpf_release(self.h, prep))

    def execute_noalloc(self, plan, out_ptr, cap, count_ptr, stream=None):
        """One plan through the fused kernel with no device allocation by
        the library; ``out_ptr`` / ``count_ptr`` are caller-owned device
        buffers (dpf_record[cap], uint32)."""
        _check(lib().dpf_execute_noalloc(self.h, C.byref(plan.plan), _stream_ptr(stream),
                                         C.c_void_p(out_ptr), int(cap), C.c_void_p(count_ptr)))

    def read_rate(self, placement="host", nbytes=1 << 31, reps=5, stream=None):
        """GB/s a kernel reads from device memory or mapped pinned host
        memory (the host-link roofline for host-resident tables)."""
        g = C.c_double()
        _check(lib().dpf_read_rate(self.h, PLACE[placement], int(nbytes), int(reps), _stream_ptr(stream),
                                   C.byref(g)))
        return g.value

    def noalloc_status(self):
        """Status word of the last allocation-free call's kernel (call after
        synchronising its stream): raises DpfError (DPF_ECORRUPT /
        DPF_EINTERNAL) when it is set, else returns 0."""
        bits = C.c_uint32()
        _check(lib().dpf_noalloc_status(self.h, C.byref(bits)))
        return bits.value

    def execute(self, plans, stream=None):
        arr = (Plan * len(plans))(*[p.plan for p in plans])
        ids = (C.c_int64 * len(plans))()
        _check(lib().dpf_execute_plan(self.h, arr, len(plans), _stream_ptr(stream), ids))
        return list(ids)

    def fetch(self, qid, timeout_ms=-1):
        n = C.c_uint64()
        cap = 1024
        while True:
            buf = np.zeros(cap, RECORD_DTYPE)
            st = lib().dpf_fetch_result(self.h, qid, _ptr(buf), cap, C.byref(n), timeout_ms)
            if st == -7:
                cap = int(n.value)
                continue
            _check(st)
            return buf[: n.value].copy()


class Server:
    """Continuous-batching request loop over a context (``dpf_server_*``):
    ``submit`` queues a plan and returns a ticket, ``wait`` returns its
    records and host times (microseconds since the server started)."""

    def __init__(self, ctx, max_batch=0, max_inflight=0, mem_budget=0, tuning=None):
        cfg = ServerConfig(max_batch, max_inflight, mem_budget, tuning or Tuning())
        h = C.c_void_p()
        _check(lib().dpf_server_create(ctx.h, C.byref(cfg), C.byref(h)))
        self.h = h
        self.ctx = ctx

    def submit(self, plan):
        t = C.c_uint64()
        _check(lib().dpf_server_submit(self.h, C.byref(plan.plan), C.byref(t)))
        return t.value

    def wait(self, ticket, timeout_ms=-1):
        n = C.c_uint64()
        times = QueryTimes()
        cap = 1024
        while True:
            buf = np.zeros(cap, RECORD_DTYPE)
            st = lib().dpf_server_wait(self.h, ticket, _ptr(buf), cap, C.byref(n), timeout_ms, C.byref(times))
            if st == -7:
                cap = int(n.value)
                continue
            _check(st)
            return buf[: n.value].copy(), {"submit_us": times.submit_us, "launch_us": times.launch_us,
                                           "done_us": times.done_us, "batch_size": times.batch_size}

    def stats(self):
        st = ServerStats()
        _check(lib().dpf_server_stats_get(self.h, C.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if self.h:
            _check(lib().dpf_server_destroy(self.h))
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def encode_column(col, page_rows=0):
    """Host encoder of the library (``dpf_encode_column``); no device work."""
    L = lib()
    codec = col["codec"]
    d = ColumnDesc(CODEC[codec], 0, int(page_rows), 0)
    P = page_rows or 65536
    if codec in STRING_CODECS:
        offs = np.ascontiguousarray(col["offsets"], np.uint64)
        data = np.ascontiguousarray(col["bytes"], np.uint8)
        values = data if data.size else np.zeros(1, np.uint8)
        n = offs.size - 1
    else:
        values = np.ascontiguousarray(col["values"], np.int64 if codec == "for64" else np.int32)
        offs = None
        n = values.size
    npages = (n + P - 1) // P
    page_off = np.zeros(npages + 1, np.uint64)
    row_prefix = np.zeros(max(npages, 1), np.uint64)
    size, dict_n = C.c_uint64(), C.c_uint64()
    _check(L.dpf_encode_column(C.byref(d), _ptr(values), _ptr(offs), n, None, 0, _ptr(page_off),
                               _ptr(row_prefix), None, 0, C.byref(dict_n), C.byref(size)))
    blob = np.zeros(size.value, np.uint8)
    dct = np.zeros(max(dict_n.value, 1), np.int32)
    _check(L.dpf_encode_column(C.byref(d), _ptr(values), _ptr(offs), n, _ptr(blob), blob.size,
                               _ptr(page_off), _ptr(row_prefix), _ptr(dct), dct.size, C.byref(dict_n),
                               C.byref(size)))
    return {"codec": codec, "rows": n, "page_rows": P, "blob": blob, "page_off": page_off,
            "row_prefix": row_prefix[:npages],
            "dict": dct[: dict_n.value] if codec in ("dict", "fsst") else None}


from .engine import Engine, PlanHandle  # noqa: E402,F401
