"""Sharded runs through the library on one GPU: the fact table's pages are
split into contiguous ranges (replicas.shard_rows), each range is loaded as
a table of its own and queried by the fused kernel (every shard builds the
same dimension tables), and the shards' int64 records, merged key by key
(replicas.merge_records), equal the oracle's records for the whole table.
This is the replica path of a multi-GPU run with the GPUs' launches taken
one after the other on one device."""

import numpy as np
import pytest

import oracle
import paper_2605_10511_gb300 as dpf
import synth
from paper_2605_10511_gb300.replicas import merge_records, shard_rows, slice_workload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world", [2, 3, 8])
def test_library_shards_merge_to_the_whole(world):
    ws = [synth.star_join(rows=(1 << 21) + 4097, seed=9, page_rows=8192),
          synth.strings(rows=(1 << 20) + 17, seed=9, page_rows=16384),
          synth.chain_join(rows=1 << 20, seed=9, page_rows=8192),
          synth.star_join(rows=(1 << 20) + 1, seed=10, page_rows=4096, bigint_measure=True),
          synth.tiny_random_workload(8, rows=30000, page_rows=1024)]
    eng = dpf.Engine(device=0)
    try:
        for w in ws:
            n = w["tables"][w["fact"]]["rows"]
            P = w["tables"][w["fact"]]["page_rows"]
            parts = []
            for r in range(world):
                lo, hi = shard_rows(n, P, r, world)
                if hi > lo:
                    parts.append(eng.run(slice_workload(w, lo, hi)))
            got = merge_records(parts, grouped=bool(w["query"]["group"]))
            want = oracle.run_query(w, from_encoded=False, threads=0)
            assert got.shape == want.shape, w["name"]
            for f in ("key", "count", "val"):
                assert np.array_equal(got[f], want[f]), (w["name"], world, f)
    finally:
        eng.close()
