"""Loader for the worked example of Sec. 2.1 (tests/golden/worked_example.txt)."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def load(path=None):
    path = path or os.path.join(HERE, "golden", "worked_example.txt")
    ex = {"param": {}, "hash": {}, "string": {}, "partition": {}, "candidate": [], "output": []}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = line.split()
        if f[0] == "param":
            ex["param"][f[1]] = int(f[2])
        elif f[0] == "hash":
            ex["hash"][f[1]] = int(f[2])
        elif f[0] == "string":
            ex["string"][int(f[1])] = f[2].encode()
        elif f[0] == "partition":
            ex["partition"][int(f[1])] = (int(f[2]), [p.encode() for p in f[3:]])
        elif f[0] in ("candidate", "output"):
            ex[f[0]].append((int(f[1]) - 1, int(f[2]) - 1))
    return ex


def table(ex, rank, bits, q, override=None):
    """Pi as an explicit table indexed by the packed rank code of a q-gram
    (first symbol most significant), from Table 2; q-grams absent from the
    table get a value above all listed ones."""
    vals = dict(ex["hash"])
    if override:
        vals.update(override)
    tab = np.full(1 << (bits * q), 10_000, dtype=np.uint64)
    for g, v in vals.items():
        code = 0
        for ch in g.encode():
            code = (code << bits) | int(rank[ch])
        tab[code] = v
    return tab
