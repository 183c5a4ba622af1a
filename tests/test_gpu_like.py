"""GPU parity of SQL LIKE ('%' any run of bytes, '_' any one byte).

General patterns run the kernel's iterative greedy wildcard matcher on STR
columns; 'p%' and '%p%' run as PREFIX / CONTAINS (also on FSST columns).
Patterns with several '%', '_' at either end, only wildcards, the empty
pattern, a pattern longer than every string; the first step and a later
step; records must equal the oracle's.  General patterns on an FSST column
are refused with DPF_EINVAL.
"""

import numpy as np
import pytest

import oracle
import paper_2605_10511_gb300 as dpf
import synth

pytestmark = pytest.mark.gpu

PATTERNS = [b"%a%b%", b"t_e%", b"%_n_%", b"%ing", b"%", b"", b"__", b"%e%e%e%", b"th%", b"%th%",
            b"q%u%", b"_%_%_", b"%" * 3 + b"x", b"a" * 32]


def assert_same(got, want, what=""):
    assert got.shape == want.shape, (what, got, want)
    for f in ("key", "count", "val"):
        assert np.array_equal(got[f], want[f]), (what, f)


@pytest.fixture(scope="module")
def eng():
    e = dpf.Engine(device=0)
    yield e
    e.close()


@pytest.mark.parametrize("later", [False, True])
def test_like_patterns_on_str(eng, later):
    w = synth.strings(rows=(1 << 17) + 33, page_rows=8192, text=True)
    eng.load_workload(w)
    for pat in PATTERNS:
        preds = [{"col": "s", "op": "like", "args": [pat]}]
        if later:  # a selective integer filter first: LIKE runs over the survivors
            preds = [{"col": "m", "op": "lt", "args": [200_000]}] + preds
        q = dict(w, query=dict(w["query"], preds=preds))
        assert_same(eng.run(q), oracle.run_query(q, from_encoded=False), (pat, later))


def test_like_on_fsst(eng):
    w = synth.strings(rows=(1 << 16) + 7, page_rows=8192, text=True, codec="fsst", contains=b"ab")
    eng.load_workload(w)
    for pat in (b"th%", b"%ing %", b"%"):
        q = dict(w, query=dict(w["query"], preds=[{"col": "s", "op": "like", "args": [pat]}]))
        assert_same(eng.run(q), oracle.run_query(q, from_encoded=False), pat)
    q = dict(w, query=dict(w["query"], preds=[{"col": "s", "op": "like", "args": [b"%a%b%"]}]))
    with pytest.raises(dpf.DpfError) as e:
        eng.run(q)
    assert e.value.status == -1
