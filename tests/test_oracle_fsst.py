"""Pins of the oracle's FSST codec and LIKE '%pattern%' predicate.

* a page worked by hand from the format definition (tests/golden/fsst_hand_worked.txt);
* round trips on edge cases: empty strings, bytes no symbol covers (escapes,
  including byte 255 itself), one-byte and long strings, a table of one symbol;
* query results are independent of the string codec (STR vs FSST) and equal
  the independent numpy evaluator, for PREFIX and CONTAINS, including an
  empty pattern (every row) and a pattern longer than every string (no row).
"""

import json
import os

import numpy as np
import pytest

import npeval
import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fsst_hand_worked.txt")


def _col(strs):
    offs = np.zeros(len(strs) + 1, np.uint64)
    np.cumsum([len(x) for x in strs], out=offs[1:])
    data = np.frombuffer(b"".join(strs), np.uint8).copy() if sum(map(len, strs)) else np.zeros(0, np.uint8)
    return {"codec": "fsst", "bytes": data, "offsets": offs}


def _table(symbols):
    t = []
    for sy in symbols:
        b = sy + b"\0" * (8 - len(sy))
        t += [int.from_bytes(b[:4], "little", signed=True), int.from_bytes(b[4:], "little", signed=True), len(sy)]
    return np.array(t, np.int32)


def _golden():
    with open(GOLDEN) as f:
        return [json.loads(x) for x in f if x.strip() and not x.startswith("#")]


@pytest.mark.parametrize("ex", _golden(), ids=lambda e: e["name"])
def test_hand_worked_fsst_page(oracle_lib, ex):
    strs = [bytes.fromhex(h) for h in ex["strings_hex"]]
    col = _col(strs)
    col["table"] = _table([bytes.fromhex(h) for h in ex["symbols_hex"]])
    enc = oracle_lib.encode_column(col, ex["page_rows"])
    assert enc["blob"].tobytes().hex() == ex["page_hex"], ex["derivation"]
    d, o = oracle_lib.decode_column(enc)
    assert d.tobytes() == b"".join(strs)


EDGE = [
    [b""],
    [b"", b"", b""],
    [b"a"],
    [bytes([255]) * 5, bytes([0, 255, 1])],
    [bytes(range(256))],
    [b"xyz" * 40],
    [b"ab" * i for i in range(60)],
]


@pytest.mark.parametrize("strs", EDGE)
def test_fsst_round_trip_edges(oracle_lib, strs):
    col = _col(strs)
    enc = oracle_lib.encode_column(col, 128)
    d, o = oracle_lib.decode_column(enc)
    assert np.array_equal(o, col["offsets"])
    assert d.tobytes() == col["bytes"].tobytes()


def test_fsst_one_symbol_table_escapes_everything_else(oracle_lib):
    col = _col([b"aaab", b"ba", b""])
    col["table"] = _table([b"aa"])
    enc = oracle_lib.encode_column(col, 128)
    d, o = oracle_lib.decode_column(enc)
    assert d.tobytes() == b"aaabba"
    assert enc["dict"].size == 3


def test_fsst_compresses_text(oracle_lib):
    w = synth.strings(rows=30000, seed=11, page_rows=8192, codec="fsst", text=True)
    c = w["tables"]["fact"]["cols"]["s"]
    enc = oracle_lib.encode_column(c, 8192)
    assert enc["blob"].size < 0.6 * c["bytes"].size
    d, o = oracle_lib.decode_column(enc)
    assert np.array_equal(d, c["bytes"]) and np.array_equal(o, c["offsets"])


@pytest.mark.parametrize("op,pat", [("prefix", b"ab"), ("contains", b"ab"), ("contains", b"q q"),
                                    ("contains", b""), ("contains", b"x" * 60), ("prefix", b"")])
@pytest.mark.parametrize("text", [False, True])
def test_string_predicates_codec_independent_and_match_numpy(oracle_lib, op, pat, text):
    ws = []
    for codec in ("str", "fsst"):
        w = synth.strings(rows=6000, seed=21, page_rows=1024, codec=codec, text=text)
        w["query"]["preds"] = [{"col": "s", "op": op, "args": [pat]}]
        ws.append(w)
    a = oracle_lib.run_query(ws[0], from_encoded=True)
    b = oracle_lib.run_query(ws[1], from_encoded=True)
    c = npeval.evaluate(ws[0])
    for f in ("key", "count", "val"):
        assert np.array_equal(a[f], b[f]) and np.array_equal(a[f], c[f]), (op, pat, f)
    if op == "contains" and pat == b"":
        assert int(a["count"].sum()) == 6000
    if len(pat) > 44:
        assert int(a["count"].sum()) == 0
