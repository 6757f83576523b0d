"""Writes the stored expected values under tests/golden/ by calling only the
FP64 oracle (oracle/).  Run from the repository root:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def four_regimes():
    """n = 4096 four-regime series, m = 128, ell = 64, k = 13: snippets for
    K = 2 and K = 4, eq. 18 criterion, the largest profile value and 64
    seeded (segment, position) cells of D."""
    s = synth.four_regimes()
    m, ell, k = 128, 64, 13
    D = oracle.profiles(s.T, m, ell, k)
    rng = np.random.default_rng(2024)
    segs = rng.integers(0, D.shape[0], size=64)
    pos = rng.integers(0, D.shape[1], size=64)
    out = {"series": "synth.four_regimes(seed=0)", "m": m, "ell": ell, "k": k,
           "S": int(D.shape[0]), "P": int(D.shape[1]), "D_max": float(D.max()),
           "row_sums": [float(x) for x in D.sum(axis=1)],
           "cells": [[int(a), int(b), float(D[a, b])] for a, b in zip(segs, pos)]}
    for K in (2, 4):
        chosen, area, labels, frac, order, _ = oracle.snippets(s.T, m, ell, k, K, D=D)
        out[f"K{K}"] = {"chosen": [int(c) for c in chosen], "area_after": [float(a) for a in area],
                        "frac": [float(f) for f in frac], "order": [int(o) for o in order],
                        "criterion": float(oracle.criterion(D, chosen)),
                        "label_counts": {str(int(c)): int((labels == c).sum()) for c in chosen}}
    return out


def tiny_full():
    """A 120-point random walk, m = 24, ell = 12, k = 3: the full profile set."""
    T = synth.white_noise(77, 120).cumsum()
    m, ell, k = 24, 12, 3
    D = oracle.profiles(T, m, ell, k)
    return {"series": "synth.white_noise(77, 120).cumsum()", "m": m, "ell": ell, "k": k,
            "D": [[float(x) for x in row] for row in D]}


if __name__ == "__main__":
    for name, fn in (("four_regimes_m128.json", four_regimes), ("tiny_walk_m24.json", tiny_full)):
        with open(os.path.join(HERE, name), "w") as f:
            json.dump(fn(), f, indent=1)
        print("wrote", name)
