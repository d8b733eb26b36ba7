"""CPU oracle for the GACE probe path -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never does.  The C source is plain single-threaded loops; this
module compiles it with gcc and marshals workload descriptions into it.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gace_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

ORC_I32, ORC_I64, ORC_F32 = 0, 1, 2
OK, EINVAL, EOVERFLOW = 0, 1, 7


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so (plain -O2, no -march)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "gace_oracle.h"))):
        tmp = _LIB + ".tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Column(C.Structure):
    _fields_ = [("dtype", C.c_int32), ("pad", C.c_int32), ("data", C.c_void_p)]


class TermS(C.Structure):
    _fields_ = [("col", C.c_uint32), ("op", C.c_uint32), ("ia", C.c_int64), ("ib", C.c_int64),
                ("fa", C.c_double), ("fb", C.c_double), ("in_off", C.c_uint32),
                ("in_len", C.c_uint32)]


class SampleS(C.Structure):
    _fields_ = [("kind", C.c_uint32), ("pad", C.c_uint32), ("block_rows", C.c_uint64),
                ("rate", C.c_double), ("seed", C.c_uint64)]


class SideS(C.Structure):
    _fields_ = [("nrows", C.c_uint64), ("cols", C.POINTER(Column)), ("ncols", C.c_uint32),
                ("key_col", C.c_uint32), ("terms", C.POINTER(TermS)), ("nterms", C.c_uint32),
                ("pad", C.c_uint32), ("in_i", C.POINTER(C.c_int64)),
                ("in_f", C.POINTER(C.c_double))]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.orc_splitmix64.restype = C.c_uint64
        L.orc_splitmix64.argtypes = [C.c_uint64]
        L.orc_hash.restype = C.c_uint64
        L.orc_hash.argtypes = [C.c_uint64, C.c_uint64]
        L.orc_threshold.restype = C.c_int
        L.orc_threshold.argtypes = [C.c_double, C.POINTER(C.c_uint64)]
        L.orc_row_in_sample.restype = C.c_int
        L.orc_row_in_sample.argtypes = [C.POINTER(SampleS), C.c_uint64]
        L.orc_probe.restype = C.c_int
        L.orc_probe.argtypes = [C.c_uint64, C.POINTER(Column), C.c_uint32, C.POINTER(SampleS),
                                C.POINTER(TermS), C.c_uint32, C.POINTER(C.c_int64),
                                C.POINTER(C.c_double), C.c_uint32, C.POINTER(C.c_uint32),
                                C.c_uint32, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64),
                                C.POINTER(C.c_uint64)]
        L.orc_selectivity.restype = C.c_double
        L.orc_selectivity.argtypes = [C.c_uint64, C.c_uint64]
        L.orc_pcs.restype = C.c_double
        L.orc_pcs.argtypes = [C.c_uint64] * 4
        L.orc_hll_registers.restype = C.c_int
        L.orc_hll_registers.argtypes = [C.c_uint64, C.POINTER(Column), C.c_uint32, C.c_uint64,
                                        C.POINTER(C.c_uint8)]
        L.orc_hll_estimate.restype = C.c_double
        L.orc_hll_estimate.argtypes = [C.POINTER(C.c_uint8), C.c_uint32]
        L.orc_ndv_exact.restype = C.c_uint64
        L.orc_ndv_exact.argtypes = [C.c_uint64, C.POINTER(Column)]
        L.orc_join_card.restype = C.c_int
        L.orc_join_card.argtypes = [C.POINTER(SideS), C.POINTER(SideS), C.c_uint64,
                                    C.POINTER(C.c_int64), C.POINTER(C.c_uint64),
                                    C.POINTER(C.c_uint64)]
        L.orc_chain_card.restype = C.c_int
        L.orc_chain_card.argtypes = [C.POINTER(SideS), C.POINTER(SideS), C.c_uint32,
                                     C.POINTER(SideS), C.c_uint64, C.c_uint64,
                                     C.POINTER(C.c_int64), C.POINTER(C.c_uint64),
                                     C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]
    return _lib


# ----------------------------------------------------------------- marshalling

_NP = {ORC_I32: np.int32, ORC_I64: np.int64, ORC_F32: np.float32}


def host_array(col, dtype_code: int) -> np.ndarray:
    """A contiguous host numpy array of the column (torch tensors are copied)."""
    if hasattr(col, "detach"):
        col = col.detach().cpu().numpy()
    return np.ascontiguousarray(np.asarray(col, dtype=_NP[dtype_code]))


class _Cols:
    def __init__(self, columns, dtypes):
        self.arrays = [host_array(c, d) for c, d in zip(columns, dtypes)]
        self.nrows = int(self.arrays[0].shape[0]) if self.arrays else 0
        self.c = (Column * max(1, len(self.arrays)))()
        for i, (a, d) in enumerate(zip(self.arrays, dtypes)):
            self.c[i].dtype = d
            self.c[i].data = a.ctypes.data_as(C.c_void_p)
        self.dtypes = list(dtypes)


class _Terms:
    """Flattened terms of one or more conjunctions plus their IN lists."""

    def __init__(self, term_lists, dtypes):
        flat = [t for lst in term_lists for t in lst]
        self.off = [0]
        for lst in term_lists:
            self.off.append(self.off[-1] + len(lst))
        ins_i, ins_f = [], []
        self.t = (TermS * max(1, len(flat)))()
        for k, t in enumerate(flat):
            s = self.t[k]
            s.col, s.op = int(t.col), int(t.op)
            is_f = t.col < len(dtypes) and dtypes[t.col] == ORC_F32
            if t.op == 2:
                s.in_off, s.in_len = len(ins_i), len(t.values)
                for v in t.values:
                    ins_i.append(int(v) if not is_f else 0)
                    ins_f.append(float(v) if is_f else 0.0)
            elif is_f:
                s.fa, s.fb = float(t.a), float(t.b)
            else:
                s.ia, s.ib = int(t.a), int(t.b)
        self.nterms = len(flat)
        self.nin = len(ins_i)
        self.in_i = np.ascontiguousarray(np.array(ins_i if ins_i else [0], dtype=np.int64))
        self.in_f = np.ascontiguousarray(np.array(ins_f if ins_f else [0.0], dtype=np.float64))

    def ptrs(self):
        return (self.in_i.ctypes.data_as(C.POINTER(C.c_int64)),
                self.in_f.ctypes.data_as(C.POINTER(C.c_double)))


def _sample(s) -> SampleS:
    out = SampleS()
    out.kind = int(s.kind)
    out.block_rows = int(s.block_rows)
    out.rate = float(s.rate)
    out.seed = int(s.seed) & ((1 << 64) - 1)
    return out


# ----------------------------------------------------------------- API

def splitmix64(x: int) -> int:
    return int(lib().orc_splitmix64(int(x) & ((1 << 64) - 1)))


def hash64(x: int, seed: int) -> int:
    return int(lib().orc_hash(int(x) & ((1 << 64) - 1), int(seed) & ((1 << 64) - 1)))


def threshold(rate: float):
    t = C.c_uint64(0)
    mode = lib().orc_threshold(float(rate), C.byref(t))
    return mode, int(t.value)


def row_in_sample(sample, row: int) -> bool:
    s = _sample(sample)
    return bool(lib().orc_row_in_sample(C.byref(s), int(row)))


class ProbeResult:
    def __init__(self, n_sample, counts, marginals):
        self.n_sample = n_sample
        self.counts = counts
        self.marginals = marginals


def probe(columns, dtypes, preds, sample, marginals: bool = True, nrows=None) -> ProbeResult:
    """counts[p] and per-term marginals of conjunctive predicates `preds`
    (a list of lists of Terms) over the rows of `sample`."""
    cols = _Cols(columns, dtypes)
    n = cols.nrows if nrows is None else int(nrows)
    terms = _Terms(preds, dtypes)
    off = np.ascontiguousarray(np.array(terms.off, dtype=np.uint32))
    counts = np.zeros(max(1, len(preds)), dtype=np.uint64)
    marg = np.zeros(max(1, terms.nterms), dtype=np.uint64)
    ns = C.c_uint64(0)
    s = _sample(sample)
    in_i, in_f = terms.ptrs()
    rc = lib().orc_probe(n, cols.c, len(cols.arrays), C.byref(s), terms.t, terms.nterms,
                         in_i, in_f, terms.nin, off.ctypes.data_as(C.POINTER(C.c_uint32)),
                         len(preds), C.byref(ns), counts.ctypes.data_as(C.POINTER(C.c_uint64)),
                         marg.ctypes.data_as(C.POINTER(C.c_uint64)) if marginals else None)
    if rc != OK:
        raise ValueError(f"oracle probe rejected its input (code {rc})")
    return ProbeResult(int(ns.value), counts[: len(preds)].copy(),
                       marg[: terms.nterms].copy() if marginals else None)


def selectivity(count: int, n: int) -> float:
    return float(lib().orc_selectivity(int(count), int(n)))


def pcs(c_ab: int, c_a: int, c_b: int, n: int) -> float:
    return float(lib().orc_pcs(int(c_ab), int(c_a), int(c_b), int(n)))


def hll_registers(column, dtype: int, p: int, seed: int) -> np.ndarray:
    cols = _Cols([column], [dtype])
    regs = np.zeros(1 << p, dtype=np.uint8)
    rc = lib().orc_hll_registers(cols.nrows, cols.c, p, int(seed) & ((1 << 64) - 1),
                                 regs.ctypes.data_as(C.POINTER(C.c_uint8)))
    if rc != OK:
        raise ValueError(f"oracle hll rejected its input (code {rc})")
    return regs


def hll_estimate(regs: np.ndarray, p: int) -> float:
    regs = np.ascontiguousarray(regs, dtype=np.uint8)
    return float(lib().orc_hll_estimate(regs.ctypes.data_as(C.POINTER(C.c_uint8)), p))


def ndv_exact(column, dtype: int) -> int:
    cols = _Cols([column], [dtype])
    return int(lib().orc_ndv_exact(cols.nrows, cols.c))


class _Side:
    def __init__(self, side):
        self.cols = _Cols(side.table.columns, side.table.dtypes)
        self.terms = _Terms([side.terms], side.table.dtypes)
        self.s = SideS()
        self.s.nrows = self.cols.nrows
        self.s.cols = self.cols.c
        self.s.ncols = len(self.cols.arrays)
        self.s.key_col = int(side.key_col)
        self.s.terms = self.terms.t
        self.s.nterms = self.terms.nterms
        self.s.in_i, self.s.in_f = self.terms.ptrs()


def join_card(fact, dim, key_domain: int):
    """(code, card, fact_pass, dim_pass) of fact JOIN dim on fact.fk = dim.key."""
    f, d = _Side(fact), _Side(dim)
    card, fp, dp = C.c_int64(0), C.c_uint64(0), C.c_uint64(0)
    rc = lib().orc_join_card(C.byref(f.s), C.byref(d.s), int(key_domain), C.byref(card),
                             C.byref(fp), C.byref(dp))
    return rc, int(card.value), int(fp.value), int(dp.value)


def chain_card(fact, dim1, dim1_fk2_col: int, dim2, key_domain1: int, key_domain2: int):
    """(code, card, fact_pass, dim1_pass, dim2_pass) of fact JOIN dim1 JOIN dim2."""
    f, d1, d2 = _Side(fact), _Side(dim1), _Side(dim2)
    card, fp, p1, p2 = C.c_int64(0), C.c_uint64(0), C.c_uint64(0), C.c_uint64(0)
    rc = lib().orc_chain_card(C.byref(f.s), C.byref(d1.s), int(dim1_fk2_col), C.byref(d2.s),
                              int(key_domain1), int(key_domain2), C.byref(card), C.byref(fp),
                              C.byref(p1), C.byref(p2))
    return rc, int(card.value), int(fp.value), int(p1.value), int(p2.value)


# ---------------------------------------------------------------- Risky Gate
# Section III-C: the three trust metrics and the paper's thresholds.
GATE_DRIFT_MIN = 0.25   # Eq. 1: D >= 0.25 triggers
GATE_SEL_ERR_MAX = 0.01  # Eq. 2: |S_est - S_probe| > 0.01 triggers
GATE_PCS_HIGH = 1.6     # Eq. 3: PCS > 1.6 (underestimation risk)
GATE_PCS_LOW = 0.7      # Eq. 3: PCS < 0.7 (overestimation risk)
RISK_DRIFT, RISK_SELECTIVITY, RISK_CORRELATION = 1, 2, 4


def gate(ndv_hist=math.nan, ndv_est=math.nan, sel_est=math.nan, sel_probe=math.nan, pcs=math.nan,
         drift_min=GATE_DRIFT_MIN, sel_err_max=GATE_SEL_ERR_MAX, pcs_high=GATE_PCS_HIGH, pcs_low=GATE_PCS_LOW):
    """(flags, D, |S_est - S_probe|) of one query's signals.  A NaN input
    leaves its signal out; D is defined only for a positive, finite NDV_hist."""
    flags, drift, sel_err = 0, math.nan, math.nan
    # Eq. 1
    if math.isfinite(ndv_hist) and ndv_hist > 0 and not math.isnan(ndv_est):
        drift = abs(ndv_hist - ndv_est) / ndv_hist
        if drift >= drift_min:
            flags |= RISK_DRIFT
    # Eq. 2
    if not math.isnan(sel_est) and not math.isnan(sel_probe):
        sel_err = abs(sel_est - sel_probe)
        if sel_err > sel_err_max:
            flags |= RISK_SELECTIVITY
    # Eq. 3
    if not math.isnan(pcs) and (pcs > pcs_high or pcs < pcs_low):
        flags |= RISK_CORRELATION
    return flags, drift, sel_err


def probe_cost(nrows, npreds, nterms, row_bytes, hashed_sets, resident, ops_per_row, alt_ms, rates):
    """Break-even model of Section V (item 2) with the measurement cost of
    Eq. 4 as kernel time: rates = dict(hbm_rate, ops_rate, h2d_rate, hash_ns,
    call_ms).  Batches of at most 32 predicates and 32 terms stream the
    referenced columns (plus one hash per row and hashed set); larger ones
    cost their compare operations.  Returns (total_ms, narrow, offload)."""
    narrow = npreds <= 32 and nterms <= 32
    if narrow:
        kernel = nrows * row_bytes / rates["hbm_rate"] * 1e3 + nrows * hashed_sets * rates["hash_ns"] * 1e-6
    else:
        ops = ops_per_row if ops_per_row > 0 else 2.0 * nterms
        kernel = nrows * ops / rates["ops_rate"] * 1e3
    transfer = 0.0 if resident else nrows * row_bytes / rates["h2d_rate"] * 1e3
    total = rates["call_ms"] + kernel + transfer
    return total, narrow, total < alt_ms
