"""Loads the page images worked by hand from the storage-format definition
(``tests/golden/hand_worked_pages.txt``): for each, the input column, the
citation, the derivation done by hand and the expected bytes of the encoded
page (Sec. 3.4.1 fixed-length layout, Sec. 3.4.2 variable-length layout,
Sec. 4.1 GPU-FOR, Sec. 4.2 page metadata); and the join chains worked by
hand from the query definition (``tests/golden/chain_hand_worked.txt``)."""

import json
import os

_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "hand_worked_pages.txt")


def _load():
    out = []
    with open(_PATH) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            e = json.loads(line)
            if "strings_hex" in e:
                e["strings"] = [bytes.fromhex(x) for x in e.pop("strings_hex")]
            out.append(e)
    return out


HAND_WORKED = _load()

_CHAIN_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "chain_hand_worked.txt")


def hand_worked_chains():
    """(workload, expected records) of the join chains worked by hand from
    the query definition in ``tests/golden/chain_hand_worked.txt``."""
    import numpy as np

    dtype = np.dtype([("key", np.int32, (2,)), ("count", np.int64), ("val", np.int64, (4,))])
    out = []
    with open(_CHAIN_PATH) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            e = json.loads(line)
            tables = {}
            for t, spec in e["tables"].items():
                cols = {c: {"codec": codec, "values": np.array(v, np.int32)} for c, (codec, v) in spec["cols"].items()}
                n = len(next(iter(spec["cols"].values()))[1])
                tables[t] = {"rows": n, "page_rows": spec["page_rows"], "cols": cols}
            w = {"name": e["name"], "tables": tables, "fact": e["fact"], "query": e["query"]}
            want = np.zeros(len(e["expect"]), dtype)
            for i, r in enumerate(e["expect"]):
                want[i]["key"] = r["key"]
                want[i]["count"] = r["count"]
                want[i]["val"][: len(r["val"])] = r["val"]
            out.append((w, want))
    return out
