"""Readers for the fixtures under tests/golden/ (inputs and expected values)."""
import json
import os

import numpy as np

from workloads import EQ, F32, I32, I64, IN, RANGE, Term

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
_OPS = {"EQ": EQ, "RANGE": RANGE, "IN": IN}
_DT = {"int32": (I32, np.int32), "int64": (I64, np.int64), "float32": (F32, np.float32)}


def _num(v, is_float):
    if is_float:
        return float(v)
    return int(v)


def load_tiny_probe():
    with open(os.path.join(GOLDEN, "tiny_probe.json")) as f:
        g = json.load(f)
    cols = g["columns"]
    dtypes = [_DT[d][0] for d in cols["dtypes"]]
    arrays = [np.array([_num(v, _DT[d][0] == F32) for v in cols[name]], dtype=_DT[d][1])
              for name, d in zip(["a", "b", "c"], cols["dtypes"])]
    preds, expect = [], []
    for p in g["predicates"]:
        terms = []
        for t in p["terms"]:
            op = _OPS[t[0]]
            c = int(t[1])
            isf = dtypes[c] == F32
            if op == IN:
                terms.append(Term(c, IN, values=tuple(_num(v, isf) for v in t[2])))
            elif op == EQ:
                terms.append(Term(c, EQ, _num(t[2], isf)))
            else:
                terms.append(Term(c, RANGE, _num(t[2], isf), _num(t[3], isf)))
        preds.append(terms)
        expect.append(p)
    return arrays, dtypes, preds, expect


def load_splitmix_vectors():
    out = []
    with open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            a, b = line.split()
            out.append((int(a, 16), int(b, 16)))
    return out
