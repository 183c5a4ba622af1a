"""Pins of the oracle's encoders and decoders (CPU only).

* hand-worked page images (closed forms, ``_hand_worked.py``);
* decode(encode(x)) == x on random data and on edge cases: constant
  columns (bw 0), the full int32 range (bw 32), sizes 1, 127, 128, 129,
  page_rows +- 1, non-monotone and wrapping deltas, empty strings;
* single-row decode through the RID index agrees with whole-column decode;
* corrupted pages are reported, not decoded.
"""

import numpy as np
import pytest

from _hand_worked import HAND_WORKED


def _column(example):
    if example["codec"] == "str":
        data = b"".join(example["strings"])
        offs = np.zeros(len(example["strings"]) + 1, np.uint64)
        offs[1:] = np.cumsum([len(s) for s in example["strings"]])
        return {"codec": "str", "bytes": np.frombuffer(data, np.uint8).copy(), "offsets": offs}
    dt = np.int64 if example["codec"] == "for64" else np.int32
    return {"codec": example["codec"], "values": np.array(example["values"], dt)}


@pytest.mark.parametrize("ex", HAND_WORKED, ids=[e["name"] for e in HAND_WORKED])
def test_hand_worked_pages(oracle_lib, ex):
    col = _column(ex)
    enc = oracle_lib.encode_column(col, ex["page_rows"])
    assert enc["page_off"].tolist() == ex["page_off"]
    assert enc["row_prefix"].tolist() == ex["row_prefix"]
    if "page_hex" in ex:
        assert enc["blob"].tobytes().hex() == ex["page_hex"]
    if "page_header_hex" in ex:
        hdr = bytes.fromhex(ex["page_header_hex"])
        assert enc["blob"][:len(hdr)].tobytes() == hdr
    if "page0_payload_prefix_hex" in ex:
        pfx = bytes.fromhex(ex["page0_payload_prefix_hex"])
        assert enc["blob"][32:32 + len(pfx)].tobytes() == pfx
    if "dict" in ex:
        assert enc["dict"].tolist() == ex["dict"]
    dec = oracle_lib.decode_column(enc)
    if ex["codec"] == "str":
        data, offs = dec
        assert data.tobytes() == b"".join(ex["strings"])
        assert offs.tolist() == col["offsets"].tolist()
    else:
        assert dec.tolist() == list(ex["values"])


def _edge_int_columns():
    rng = np.random.default_rng(7)
    i32 = np.iinfo(np.int32)
    cases = {
        "one": np.array([42], np.int32),
        "const_127": np.full(127, -3, np.int32),
        "full_range_128": np.array([i32.min, i32.max] * 64, np.int32),
        "full_range_129": rng.integers(i32.min, i32.max, 129, dtype=np.int64, endpoint=True).astype(np.int32),
        "extremes_only": np.array([i32.max, i32.min, i32.min, i32.max, 0], np.int32),
        "small_random": rng.integers(-5, 5, 1000, dtype=np.int32),
        "wide_random": rng.integers(i32.min, i32.max, 5000, dtype=np.int64, endpoint=True).astype(np.int32),
        "sorted": np.sort(rng.integers(0, 1 << 20, 3000, dtype=np.int32)),
        "descending": np.sort(rng.integers(-100000, 100000, 2000, dtype=np.int32))[::-1].copy(),
        "sawtooth": (np.arange(3000, dtype=np.int32) % 300) * 1000 - 7,
    }
    return cases


@pytest.mark.parametrize("codec", ["for", "delta", "dict"])
@pytest.mark.parametrize("page_rows", [128, 256, 1024])
def test_roundtrip_int_edges(oracle_lib, codec, page_rows):
    for name, v in _edge_int_columns().items():
        if codec == "dict" and np.unique(v).size > 65536:
            continue
        for n in sorted({v.size, min(v.size, page_rows - 1), min(v.size, page_rows + 1)}):
            x = v[:n]
            enc = oracle_lib.encode_column({"codec": codec, "values": x}, page_rows)
            dec = oracle_lib.decode_column(enc)
            assert np.array_equal(dec, x), (name, n)
            # the RID index is the inclusive prefix of page row counts
            npages = (n + page_rows - 1) // page_rows
            expect_prefix = [min(n, (p + 1) * page_rows) for p in range(npages)]
            assert enc["row_prefix"].tolist() == expect_prefix
            # pages start on 16-byte boundaries
            assert all(int(o) % 16 == 0 for o in enc["page_off"])


def test_bit_widths_are_minimal(oracle_lib):
    """bw = bits of (max - min): a span of 2^k - 1 needs k bits, 2^k needs k+1."""
    for k in range(0, 32):
        for span in {(1 << k) - 1, 1 << k} if k < 31 else {(1 << k) - 1}:
            v = np.zeros(128, np.int64)
            v[5] = span
            v = (v - (1 << 30)).astype(np.int32)
            enc = oracle_lib.encode_column({"codec": "for", "values": v}, 128)
            wob = int(np.frombuffer(enc["blob"][20:24].tobytes(), np.uint32)[0])
            assert wob & 0xFF == int(span).bit_length(), span
            assert np.array_equal(oracle_lib.decode_column(enc), v)


def _edge_int64_columns():
    i64 = np.iinfo(np.int64)
    rng = np.random.default_rng(11)
    return {
        "one": np.array([-(1 << 40)], np.int64),
        "full_range_128": np.array([i64.min, i64.max] * 64, np.int64),
        "full_range_random": rng.integers(i64.min, i64.max, 1000, dtype=np.int64, endpoint=True),
        "extremes_ragged": np.array([i64.max, i64.min, 0, -1, 1, i64.max - 1, i64.min + 1], np.int64),
        "wide_cents": rng.integers(0, 1 << 44, 3000, dtype=np.int64) - (1 << 43),
        "int32_like": rng.integers(-5, 5, 700, dtype=np.int64),
        "constant": np.full(300, 1 << 50, np.int64),
    }


@pytest.mark.parametrize("page_rows", [128, 256, 1024])
def test_roundtrip_for64_edges(oracle_lib, page_rows):
    for name, v in _edge_int64_columns().items():
        for n in sorted({v.size, min(v.size, page_rows - 1), min(v.size, page_rows + 1)}):
            x = v[:n]
            enc = oracle_lib.encode_column({"codec": "for64", "values": x}, page_rows)
            assert np.array_equal(oracle_lib.decode_column(enc), x), (name, n)
            for r in {0, n // 2, n - 1}:
                assert oracle_lib.decode_row(enc, r) == int(x[r]), (name, n, r)
            assert all(int(o) % 16 == 0 for o in enc["page_off"])


def test_for64_bit_widths_are_minimal_and_pages_sized(oracle_lib):
    """bw = bits of (max - min) for every width 0..64, and a page holds the
    16-byte header, 16 bytes per mini block header (rounded to 16) and 2*bw
    words of 8 bytes per mini block."""
    for k in range(0, 65):
        span = (1 << k) - 1
        v = np.full(128, -(1 << 63), np.int64)
        v[77] = np.int64(np.uint64(span).astype(np.int64)) + v[0] if k < 64 else np.iinfo(np.int64).max
        enc = oracle_lib.encode_column({"codec": "for64", "values": v}, 128)
        bw = int(np.frombuffer(enc["blob"][28:32].tobytes(), np.uint32)[0])
        assert bw == k, (k, bw)
        assert enc["page_off"].tolist() == [0, 32 + 16 * k], k
        assert np.array_equal(oracle_lib.decode_column(enc), v)


def test_delta_wraps_modulo_2_32(oracle_lib):
    i32 = np.iinfo(np.int32)
    v = np.array([i32.max, i32.min, i32.max, 0, i32.min, -1, 1], np.int32)
    enc = oracle_lib.encode_column({"codec": "delta", "values": v}, 128)
    assert np.array_equal(oracle_lib.decode_column(enc), v)


@pytest.mark.parametrize("page_rows", [128, 384])
def test_roundtrip_strings(oracle_lib, page_rows):
    rng = np.random.default_rng(3)
    for n in [1, 127, 128, 129, page_rows - 1, page_rows + 1, 3 * page_rows + 5]:
        lens = rng.integers(0, 50, n)
        lens[rng.integers(0, n, max(1, n // 10))] = 0
        offs = np.zeros(n + 1, np.uint64)
        offs[1:] = np.cumsum(lens)
        data = rng.integers(0, 256, int(offs[-1]), dtype=np.uint8)
        enc = oracle_lib.encode_column({"codec": "str", "bytes": data, "offsets": offs}, page_rows)
        d2, o2 = oracle_lib.decode_column(enc)
        assert np.array_equal(o2, offs)
        assert np.array_equal(d2, data)


def test_row_decode_matches_column_decode(oracle_lib):
    rng = np.random.default_rng(11)
    v = rng.integers(-1000, 1000, 1000, dtype=np.int32)
    v[300:500] = np.sort(v[300:500])
    for codec in ["for", "delta", "dict"]:
        enc = oracle_lib.encode_column({"codec": codec, "values": v}, 256)
        full = oracle_lib.decode_column(enc)
        for r in [0, 1, 127, 128, 255, 256, 257, 511, 999] + list(rng.integers(0, 1000, 40)):
            assert oracle_lib.decode_row(enc, int(r)) == int(full[r]) == int(v[r])


def test_corrupted_pages_are_reported(oracle_lib):
    v = np.arange(1000, dtype=np.int32)
    enc = oracle_lib.encode_column({"codec": "for", "values": v}, 256)
    bad = dict(enc)
    bad["blob"] = enc["blob"].copy()
    bad["blob"][0] ^= 0xFF        # magic
    with pytest.raises(oracle_lib.OracleError):
        oracle_lib.decode_column(bad)
    bad["blob"] = enc["blob"].copy()
    bad["blob"][20] = 40          # bit width 40 > 32
    with pytest.raises(oracle_lib.OracleError):
        oracle_lib.decode_column(bad)
    # wrong codec for the page
    other = dict(enc)
    other["codec"] = "delta"
    with pytest.raises(oracle_lib.OracleError):
        oracle_lib.decode_column(other)
