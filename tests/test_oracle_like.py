"""The oracle's SQL LIKE (CPU only): '%' = any run of bytes, '_' = any one
byte, the whole string against the whole pattern, no escape character.

Pinned by cases worked by hand, by Python's regular-expression engine on
random strings and patterns (an independent matcher), and by queries whose
LIKE reduces to the PREFIX / CONTAINS predicates already pinned ('p%',
'%p%').  Planted mistakes in a copy of the oracle are caught.
"""

import os
import random
import re
import subprocess
import tempfile

import numpy as np
import pytest

import npeval
import oracle
import synth

# (string, pattern, matches) worked by hand
HAND_WORKED = [
    (b"", b"", True), (b"", b"%", True), (b"", b"_", False), (b"a", b"", False),
    (b"abc", b"abc", True), (b"abc", b"ab", False), (b"abc", b"a%", True), (b"abc", b"%c", True),
    (b"abc", b"%b%", True), (b"abc", b"a_c", True), (b"abc", b"a__c", False), (b"abc", b"___", True),
    (b"abc", b"____", False), (b"abc", b"%%%", True), (b"abc", b"a%b%c", True), (b"abc", b"a%c%b", False),
    (b"aaa", b"a%a%a", True), (b"aa", b"a%a%a", False), (b"mississippi", b"m%iss%ppi", True),
    (b"mississippi", b"%s_s%", True), (b"mississippi", b"%ss_ss%", True), (b"mississippi", b"%ss__ss%", False),
    (b"hello world", b"% w%", True),
    (b"hello world", b"h%o%o%", True), (b"hello world", b"h%o%o%x", False), (b"abab", b"%ab", True),
    (b"abab", b"_b%b", True), (b"abab", b"%b_", False),
]


def _table(strings):
    offs = np.zeros(len(strings) + 1, np.uint64)
    offs[1:] = np.cumsum([len(x) for x in strings])
    data = np.frombuffer(b"".join(strings), np.uint8).copy() if any(strings) else np.zeros(0, np.uint8)
    return {"codec": "str", "bytes": data, "offsets": offs}


def _workload(strings, pattern):
    n = len(strings)
    return {"name": "like", "fact": "f", "tables": {"f": {"rows": n, "page_rows": 128, "cols": {
        "s": _table(strings), "m": {"codec": "for", "values": np.arange(n, dtype=np.int32)}}}},
        "query": {"preds": [{"col": "s", "op": "like", "args": [pattern]}], "joins": [], "group": [],
                  "aggs": [{"op": "sum", "cols": ["m"]}]}}


def _oracle_rows(strings, pattern, o=oracle):
    """The rows the oracle keeps, recovered from SUM(2^r) over r < 60."""
    out = o.run_query(_workload(strings, pattern), from_encoded=False)
    return int(out["count"][0]), int(out["val"][0][0])


def _run_hand_worked(o):
    for s, p, m in HAND_WORKED:
        cnt, _ = _oracle_rows([s], p, o)
        assert cnt == int(m), (s, p, m)


def test_hand_worked_cases(oracle_lib):
    _run_hand_worked(oracle)


def _random_cases(seed, n=400):
    rng = random.Random(seed)
    strings = [bytes(rng.choice(b"ab ") for _ in range(rng.randrange(0, 9))) for _ in range(n)]
    pats = [bytes(rng.choice(b"ab %_") for _ in range(rng.randrange(0, 7))) for _ in range(40)]
    return strings, pats


def test_random_against_regex(oracle_lib):
    for seed in range(5):
        strings, pats = _random_cases(seed)
        for p in pats:
            rx = re.compile(b"".join(b".*" if c == 0x25 else b"." if c == 0x5F else re.escape(bytes([c]))
                                     for c in p), re.DOTALL)
            want = [i for i, s in enumerate(strings) if rx.fullmatch(s)]
            w = _workload(strings, p)
            out = oracle.run_query(w, from_encoded=False)
            assert int(out["count"][0]) == len(want), (seed, p)
            assert int(out["val"][0][0]) == sum(want), (seed, p)


def test_like_reduces_to_prefix_and_contains(oracle_lib):
    w = synth.strings(rows=20_000, page_rows=4096, text=True)
    for pat in (b"th", b"e a", b"q"):
        for like, op in ((pat + b"%", "prefix"), (b"%" + pat + b"%", "contains")):
            a = dict(w, query=dict(w["query"], preds=[{"col": "s", "op": "like", "args": [like]}]))
            b = dict(w, query=dict(w["query"], preds=[{"col": "s", "op": op, "args": [pat]}]))
            ra, rb = oracle.run_query(a, from_encoded=False), oracle.run_query(b, from_encoded=False)
            assert np.array_equal(ra, rb), (like, op)


def test_numpy_evaluator_agrees_on_text(oracle_lib):
    w = synth.strings(rows=5_000, page_rows=1024, text=True)
    for pat in (b"%a%b%", b"t_e%", b"%_n_%", b"%ing", b"%"):
        q = dict(w, query=dict(w["query"], preds=[{"col": "s", "op": "like", "args": [pat]}]))
        got, want = oracle.run_query(q, from_encoded=False), npeval.evaluate(q)
        assert got.shape == want.shape and np.array_equal(got["count"], want["count"]), pat


ORACLE_SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "dpf_oracle.cpp")
MUTANTS = {
    "percent_never_empty": ("if (p[j - 1] == '%') m[i][j] = m[i][j - 1] || m[i - 1][j];",
                            "if (p[j - 1] == '%') m[i][j] = m[i - 1][j - 1] || m[i - 1][j];"),
    "underscore_literal": ("(p[j - 1] == '_' || p[j - 1] == s[i - 1])", "(p[j - 1] == s[i - 1])"),
    "empty_pattern_prefix": ("m[0][j] = p[j - 1] == '%' && m[0][j - 1];", "m[0][j] = p[j - 1] == '%';"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_like_mutant_is_caught(oracle_lib, name):
    old, new = MUTANTS[name]
    src = open(ORACLE_SRC).read()
    assert src.count(old) == 1, name
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "m.cpp")
        open(path, "w").write(src.replace(old, new))
        so = os.path.join(tmp, "libm.so")
        subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-pthread", "-o", so, path])
        caught = False
        with oracle.use_library(so):
            try:
                _run_hand_worked(oracle)
                for seed in range(3):
                    strings, pats = _random_cases(seed, 200)
                    for p in pats:
                        rx = re.compile(b"".join(b".*" if c == 0x25 else b"." if c == 0x5F else re.escape(bytes([c]))
                                                 for c in p), re.DOTALL)
                        assert _oracle_rows(strings, p)[0] == sum(1 for s in strings if rx.fullmatch(s))
            except AssertionError:
                caught = True
        assert caught, name
