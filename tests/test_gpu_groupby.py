"""GPU parity of the warp-aggregated group-by (hash aggregation of Kernel #3).

The lanes of a round that hold the same group id add their values once
(their peers found by __match_any_sync, the group's lowest lane issuing the
atomic).  The cases that exercise it most: every row passing a filter with
Zipf-skewed keys (the top key holds about a fifth of the rows), one hot
group holding almost every row, groups in shared-memory and in global
accumulators, each with warp aggregation and with one atomic per row (the
two group_agg tunings), COUNT / SUM / SUM_MUL / SUM_SUB over 32- and 64-bit operands,
ragged tails.  Records must equal the oracle's exactly.
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


@pytest.mark.parametrize("rows", [(1 << 21) + 333, 1 << 25])
def test_all_rows_pass_with_zipf_keys(eng, rows):
    """An empty prefix keeps every row: 1,024 Zipf(1.1) groups take all of
    them (the full 2^25-row strings table in the bench's configuration)."""
    w = synth.strings(rows=rows, prefix=b"")
    want = oracle.run_query(w, from_encoded=False, threads=0)
    assert int(want["count"].sum()) == rows
    assert int(want["count"].max()) > rows // 8  # the Zipf head: many lanes of a round share it
    for mode in ("atomic", "warp"):
        t = dpf.Tuning(0, 0, 0, 0, 0, dpf.GROUP_AGG[mode])
        assert_same(eng.run(w, tuning=t), want, (w["name"], mode))


@pytest.mark.parametrize("n_groups,hot_frac", [(1, 0.0), (5, 0.97), (300, 0.5), (20000, 0.3)])
def test_hot_groups_and_wide_sums(eng, n_groups, hot_frac):
    """One key holding most rows (up to all 32 lanes of a round in one
    group), int32 and int64 (FOR64) operands, products and differences that
    wrap modulo 2^64; 20,000 x 3 groups exceed the shared accumulators and
    run on global ones."""
    w = synth.hot_groups(300_001, n_groups, hot_frac, seed=n_groups)
    want = oracle.run_query(w, from_encoded=False)
    for mode in ("atomic", "warp"):
        for threads in (256, 1024):
            t = dpf.Tuning(2048, threads, 0, 0, 0, dpf.GROUP_AGG[mode])
            assert_same(eng.run(w, tuning=t), want, (w["name"], mode, threads))
