"""C ABI and host logic of the CUDA library, on the CPU (no GPU compute).

* the library builds and exports every function ``include/dpf.h`` declares;
* the library's host encoder (the data loader) writes exactly the bytes of
  the oracle's independent encoder, for every codec, edge case and page size;
* argument errors are reported as statuses with a message;
* without a GPU, creating a context fails loudly (no CPU fallback).
"""

import os
import re
import subprocess

import numpy as np
import pytest

import paper_2605_10511_gb300 as dpf
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(dpf_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    path = dpf.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (dpf_[a-z0-9_]+)\b", out))
    declared = _declared_functions()
    assert declared, "no declarations found"
    missing = declared - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    L = dpf.lib()
    for name in declared:
        assert getattr(L, name) is not None


def test_binding_covers_every_declared_symbol():
    assert _declared_functions() == set(dpf._SIGS)


def _compare(col, page_rows):
    import oracle
    a = dpf.encode_column(col, page_rows)
    if col["codec"] == "fsst":
        # the two FSST encoders choose their symbol tables independently; the
        # library's pages must decode, with the oracle's decoder, to the input
        d, o = oracle.decode_column(a)
        assert np.array_equal(o, np.asarray(col["offsets"], np.uint64) - np.uint64(col["offsets"][0]))
        assert d.tobytes() == np.asarray(col["bytes"], np.uint8).tobytes()
        return
    b = oracle.encode_column(col, page_rows)
    assert a["blob"].tobytes() == b["blob"].tobytes()
    assert np.array_equal(a["page_off"], b["page_off"])
    assert np.array_equal(a["row_prefix"], b["row_prefix"])
    if col["codec"] == "dict":
        assert np.array_equal(a["dict"], b["dict"])


@pytest.mark.parametrize("seed", range(25))
def test_encoder_matches_oracle_on_random_tables(oracle_lib, seed):
    w = synth.tiny_random_workload(seed)
    for t in w["tables"].values():
        for c in t["cols"].values():
            _compare(c, t["page_rows"])


@pytest.mark.parametrize("codec", ["for", "delta", "dict"])
def test_encoder_matches_oracle_on_edges(oracle_lib, codec):
    rng = np.random.default_rng(5)
    i32 = np.iinfo(np.int32)
    cases = [np.array([7], np.int32), np.full(129, -1, np.int32),
             np.array([i32.min, i32.max] * 100, np.int32),
             rng.integers(i32.min, i32.max, 3000, dtype=np.int64, endpoint=True).astype(np.int32),
             np.sort(rng.integers(0, 10**6, 5000)).astype(np.int32)]
    for v in cases:
        if codec == "dict" and np.unique(v).size > 65536:
            continue
        for P in (128, 256, 4096):
            _compare({"codec": codec, "values": v}, P)


def test_for64_encoder_matches_oracle_on_edges(oracle_lib):
    rng = np.random.default_rng(9)
    i64 = np.iinfo(np.int64)
    cases = [np.array([-(1 << 40)], np.int64), np.full(129, 1 << 50, np.int64),
             np.array([i64.min, i64.max] * 100, np.int64),
             rng.integers(i64.min, i64.max, 3000, dtype=np.int64, endpoint=True),
             rng.integers(0, 1 << 44, 5000, dtype=np.int64) - (1 << 43)]
    for k in range(65):  # every bit width 0..64 in one mini block each
        v = np.zeros(128, np.int64)
        v[3] = np.int64(np.uint64((1 << k) - 1).astype(np.int64)) if k < 64 else np.int64(-1)
        v[5] = i64.min if k == 64 else 0
        cases.append(v)
    for v in cases:
        for P in (128, 256, 4096):
            _compare({"codec": "for64", "values": v}, P)


def test_encoder_matches_oracle_on_workload_columns(oracle_lib):
    for w in (synth.scan_filter_aggregate(rows=300000, page_rows=65536),
              synth.strings(rows=100000, page_rows=8192),
              synth.chain_join(rows=1 << 17, page_rows=16384),
              synth.star_join(rows=150000, dim_rows=(2000, 30000, 20000), clustered=True,
                              bigint_measure=True)):
        for t in w["tables"].values():
            for c in t["cols"].values():
                _compare(c, t["page_rows"])


def test_encoder_argument_errors():
    with pytest.raises(dpf.DpfError) as e:
        dpf.encode_column({"codec": "for", "values": np.zeros(10, np.int32)}, 100)
    assert e.value.status == -1 and "page_rows" in str(e.value)
    with pytest.raises(dpf.DpfError):
        dpf.encode_column({"codec": "dict", "values": np.arange(70000, dtype=np.int32)}, 128)
    with pytest.raises(dpf.DpfError):
        dpf.encode_column({"codec": "for", "values": np.zeros(0, np.int32)}, 128)


def test_no_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(dpf.DpfError) as e:
        dpf.Context(0)
    assert e.value.status == -3


@pytest.mark.parametrize("text", [False, True])
def test_library_fsst_pages_decode_with_the_oracle(oracle_lib, text):
    """The library's FSST encoder (its own symbol table) writes pages that the
    oracle's independent decoder turns back into the same strings."""
    import synth
    w = synth.strings(rows=9000, seed=5, page_rows=2048, codec="fsst", text=text)
    c = w["tables"]["fact"]["cols"]["s"]
    enc = dpf.encode_column(c, 2048)
    assert enc["dict"] is not None and enc["dict"].size % 3 == 0 and 0 < enc["dict"].size <= 765
    d, o = oracle_lib.decode_column(enc)
    assert np.array_equal(o, c["offsets"]) and np.array_equal(d, c["bytes"])
    if text:
        assert enc["blob"].size < 0.6 * c["bytes"].size


@pytest.mark.parametrize("strs", [[b""], [b"", b"a", b""], [bytes(range(256)) * 2], [b"\\xff" * 40]])
def test_library_fsst_edges_decode_with_the_oracle(oracle_lib, strs):
    offs = np.zeros(len(strs) + 1, np.uint64)
    np.cumsum([len(x) for x in strs], out=offs[1:])
    data = np.frombuffer(b"".join(strs), np.uint8).copy()
    col = {"codec": "fsst", "bytes": data, "offsets": offs}
    enc = dpf.encode_column(col, 128)
    d, o = oracle_lib.decode_column(enc)
    assert np.array_equal(o, offs) and d.tobytes() == b"".join(strs)
