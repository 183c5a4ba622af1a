"""GPU parity of LIKE on FSST-compressed strings matched code by code.

With the join-table placement that keeps tables in shared memory (AUTO or
SMEM), a PREFIX / CONTAINS step on an FSST column runs the matcher one
symbol code at a time through tables the CTA builds from the column's
symbol table (next state after each symbol and after each escaped byte);
with GLOBAL placement it decodes byte by byte.  Patterns of 1..32 bytes,
with self-overlaps that exercise the automaton's fall-backs (aab, abab),
patterns that span symbol boundaries, absent patterns and prefixes longer
than strings: both ways must give the oracle's records.
"""

import numpy as np
import pytest

import oracle
import paper_2605_10511_gb300 as dpf
import synth

pytestmark = pytest.mark.gpu


def assert_same(got, want, what=""):
    assert got.shape == want.shape, (what, got, want)
    for f in ("key", "count", "val"):
        assert np.array_equal(got[f], want[f]), (what, f)


@pytest.fixture(scope="module")
def eng():
    e = dpf.Engine(device=0)
    yield e
    e.close()


@pytest.fixture(scope="module")
def text():
    return synth.strings(rows=(1 << 18) + 91, page_rows=16384, text=True, codec="fsst", contains=b"ab")


PATTERNS = [b"e", b"ab", b"th", b"the ", b"aab", b"abab", b"ing t", b"zzzq", b" a", b"tion", b"qu",
            b"an the", b"a" * 5, b"xyzxyzxyzxyzxyzxyzxyzxyzxyzxyzxy"]


@pytest.mark.parametrize("op", ["contains", "prefix"])
@pytest.mark.parametrize("place", ["auto", "global"])
def test_fsst_like_patterns(eng, text, op, place):
    eng.load_workload(text)
    t = dpf.Tuning(0, 256, dpf.HT_PLACE[place], 0)
    for pat in PATTERNS:
        w = dict(text)
        w["query"] = dict(text["query"], preds=[{"col": "s", "op": op, "args": [pat]}])
        want = oracle.run_query(w, from_encoded=False)
        assert_same(eng.run(w, tuning=t), want, (op, place, pat))
