"""Loads the page images worked by hand from the storage-format definition
(``tests/golden/hand_worked_pages.txt``): for each, the input column, the
citation, the derivation done by hand and the expected bytes of the encoded
page (Sec. 3.4.1 fixed-length layout, Sec. 3.4.2 variable-length layout,
Sec. 4.1 GPU-FOR, Sec. 4.2 page metadata)."""

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
