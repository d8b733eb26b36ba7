"""Python binding of libgace, the GB300 probe engine of GACE (arXiv 2512.19750).

Same names as the C ABI (include/gace.h); this layer only marshals Python
descriptions (workloads.Term / workloads.Sample, torch tensors, numpy arrays)
into the C structures.  Every step of the probe runs in the library's CUDA
kernels: nothing here computes a result, and there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _capi
from ._capi import (GACE_BLOCKS, GACE_BORROW, GACE_COPY, GACE_EBUSY, GACE_ECUDA, GACE_EINVAL, GACE_ENOMEM,
                    GACE_ENOTFOUND, GACE_EOVERFLOW, GACE_EPENDING, GACE_EQ, GACE_ETIMEDOUT,
                    GACE_F32, GACE_FULL, GACE_I32,
                    GACE_I64, GACE_IN, GACE_JOIN_AUTO, GACE_JOIN_GATHER, GACE_JOIN_HIST_DOT,
                    GACE_OK, GACE_RANGE, GACE_REQ_JOIN, GACE_REQ_NDV, GACE_REQ_PROBE, GACE_ROWS,
                    GACE_RISK_CORRELATION, GACE_RISK_DRIFT, GACE_RISK_SELECTIVITY, GaceError, check, lib)

RESULT_DTYPE = np.dtype([("match", "<u8"), ("sample_rows", "<u8"), ("sel", "<f8"), ("pcs", "<f8")])
_NP_OF = {GACE_I32: np.int32, GACE_I64: np.int64, GACE_F32: np.float32}


def _dtype_code(x) -> int:
    name = str(getattr(x, "dtype", x))
    if "int32" in name:
        return GACE_I32
    if "int64" in name:
        return GACE_I64
    if "float32" in name:
        return GACE_F32
    raise ValueError(f"unsupported column dtype {name}")


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


# ----------------------------------------------------------------- marshalling

class TermBatch:
    """C arrays of a predicate batch: gace_term, gace_pred and in_values."""

    def __init__(self, preds, dtypes):
        flat = [t for p in preds for t in p]
        self.nterms = len(flat)
        self.npreds = len(preds)
        self.terms = (_capi.gace_term * max(1, self.nterms))()
        self.preds = (_capi.gace_pred * max(1, self.npreds))()
        ins = []
        for k, t in enumerate(flat):
            s = self.terms[k]
            s.col, s.op = int(t.col), int(t.op)
            isf = 0 <= t.col < len(dtypes) and dtypes[t.col] == GACE_F32
            if t.op == GACE_IN:
                s.in_off, s.in_len = len(ins), len(t.values)
                ins.extend((isf, v) for v in t.values)
            elif isf:
                s.a.f, s.b.f = float(t.a), float(t.b)
            else:
                s.a.i, s.b.i = int(t.a), int(t.b)
        self.nin = len(ins)
        self.in_values = (_capi.gace_scalar * max(1, self.nin))()
        for k, (isf, v) in enumerate(ins):
            if isf:
                self.in_values[k].f = float(v)
            else:
                self.in_values[k].i = int(v)
        off = 0
        for k, p in enumerate(preds):
            self.preds[k].term_off, self.preds[k].term_cnt = off, len(p)
            off += len(p)


def _samples(samples):
    arr = (_capi.gace_sample * max(1, len(samples)))()
    for k, s in enumerate(samples):
        arr[k].kind = int(s.kind)
        arr[k].block_rows = int(s.block_rows)
        arr[k].rate = float(s.rate)
        arr[k].seed = int(s.seed) & ((1 << 64) - 1)
    return arr


# ----------------------------------------------------------------- ABI wrappers

def gace_abi_version() -> int:
    return int(lib().gace_abi_version())


def gace_create(device: int = 0, stream=None, hbm_budget_bytes: int = 0,
                wait_timeout_ms: int = 0, max_ctas: int = 0, rank_min_rows: int = 0,
                rank_search: int = 0) -> int:
    cfg = _capi.gace_config(device, wait_timeout_ms, hbm_budget_bytes, _stream_handle(stream), max_ctas,
                            rank_min_rows, rank_search)
    out = C.c_void_p()
    check(lib().gace_create(C.byref(out), C.byref(cfg)), "gace_create")
    return out.value


def gace_destroy(ctx) -> None:
    """Frees the context; a running scheduler first finishes its requests."""
    check(lib().gace_destroy(ctx), "gace_destroy")
    for key in [k for k in _SUBMITTED if k[0] == _ctx_key(ctx)]:
        del _SUBMITTED[key]
    for key in [k for k in _LAZY_KEEP if k[0] == _ctx_key(ctx)]:
        del _LAZY_KEEP[key]


def gace_load_columns(ctx, columns, borrow: bool = False, copy_on_first_probe: bool = False) -> int:
    """Registers a table; columns are torch tensors (CUDA or CPU) or numpy
    arrays, all of one length.  borrow=True keeps the device pointers;
    copy_on_first_probe=True (host columns) defers the copy to the first call
    that reads the table, which a probe overlaps with its passes (the columns
    must stay alive and unchanged until then)."""
    n = len(columns)
    arr = (_capi.gace_column * n)()
    keep = []
    nrows = None
    for k, c in enumerate(columns):
        if hasattr(c, "data_ptr"):
            if not c.is_contiguous():
                raise ValueError("column tensors must be contiguous")
            arr[k].dtype = _dtype_code(c.dtype)
            arr[k].on_device = 1 if c.is_cuda else 0
            arr[k].data = c.data_ptr() if c.numel() else None
            rows = int(c.shape[0])
        else:
            a = np.ascontiguousarray(c)
            keep.append(a)
            arr[k].dtype = _dtype_code(a.dtype)
            arr[k].on_device = 0
            arr[k].data = a.ctypes.data if a.size else None
            rows = int(a.shape[0])
        if nrows is None:
            nrows = rows
        elif rows != nrows:
            raise ValueError("columns differ in length")
    if any(getattr(c, "is_cuda", False) for c in columns):
        import torch

        # the library reads the columns on its own stream: what torch queued to
        # produce them must have finished
        torch.cuda.synchronize()
    tid = C.c_uint32()
    flags = GACE_BORROW if borrow else (_capi.GACE_COPY_ON_FIRST_PROBE if copy_on_first_probe else GACE_COPY)
    check(lib().gace_load_columns(ctx, nrows or 0, n, arr, flags,
                                  C.byref(tid)), "gace_load_columns")
    if copy_on_first_probe:  # the library copies them later: keep them alive until the unload
        _LAZY_KEEP[(_ctx_key(ctx), int(tid.value))] = (keep, list(columns))
    return int(tid.value)


_LAZY_KEEP: dict = {}  # (context, table) -> host columns a deferred copy still reads


def gace_unload(ctx, table_id: int) -> None:
    check(lib().gace_unload(ctx, table_id), "gace_unload")
    _LAZY_KEEP.pop((_ctx_key(ctx), int(table_id)), None)


def gace_probe_batch(ctx, table_id: int, preds, samples, dtypes, marginals: bool = False,
                     batch: TermBatch | None = None):
    """Counts of conjunctive predicates on each row set.

    Returns (results, term_marginals): results is a structured array of shape
    (len(samples), len(preds)) with fields match, sample_rows, sel, pcs;
    term_marginals is (len(samples), nterms) uint64 or None."""
    b = batch or TermBatch(preds, dtypes)
    smp = _samples(samples)
    res = np.zeros((len(samples), b.npreds), dtype=RESULT_DTYPE)
    marg = np.zeros((len(samples), b.nterms), dtype=np.uint64) if marginals else None
    rc = lib().gace_probe_batch(
        ctx, table_id, smp, len(samples), b.terms, b.nterms, b.in_values, b.nin, b.preds, b.npreds,
        res.ctypes.data_as(C.POINTER(_capi.gace_pred_result)),
        marg.ctypes.data_as(C.POINTER(C.c_uint64)) if marginals and b.nterms else None)
    check(rc, "gace_probe_batch")
    return res, marg


def gace_ndv(ctx, table_id: int, col: int, p: int, hash_seed: int):
    """(registers uint8[2^p], estimate) of HyperLogLog on one column."""
    regs = np.zeros(1 << p, dtype=np.uint8)
    est = C.c_double()
    check(lib().gace_ndv(ctx, table_id, col, p, int(hash_seed) & ((1 << 64) - 1),
                         regs.ctypes.data_as(C.POINTER(C.c_uint8)), C.byref(est)), "gace_ndv")
    return regs, float(est.value)


def gace_ndv_noalloc(column, p: int, hash_seed: int, stream=None):
    """(registers uint8[2^p], estimate) of one CUDA tensor column through the
    no-allocation entry point (no context; fixed scratch inside the library)."""
    if not (hasattr(column, "is_cuda") and column.is_cuda and column.is_contiguous()):
        raise ValueError("column must be a contiguous CUDA tensor")
    regs = np.zeros(1 << p, dtype=np.uint8)
    est = C.c_double()
    check(lib().gace_ndv_noalloc(column.data_ptr() if column.numel() else None, _dtype_code(column.dtype),
                                 column.numel(), p, int(hash_seed) & ((1 << 64) - 1),
                                 _stream_handle(stream), regs.ctypes.data_as(C.POINTER(C.c_uint8)),
                                 C.byref(est)), "gace_ndv_noalloc")
    return regs, float(est.value)


class JoinSideSpec:
    """(table_id, key column, filter terms, column dtypes) of one join side."""

    def __init__(self, table_id: int, key_col: int, terms=(), dtypes=()):
        self.table_id, self.key_col = table_id, key_col
        self.batch = TermBatch([list(terms)], list(dtypes))

    def fill(self, s: _capi.gace_join_side):
        s.table_id, s.key_col = self.table_id, self.key_col
        s.terms = C.cast(self.batch.terms, C.POINTER(_capi.gace_term))
        s.nterms = self.batch.nterms
        s.in_values = C.cast(self.batch.in_values, C.POINTER(_capi.gace_scalar))
        s.nin = self.batch.nin


def gace_join_card(ctx, fact: JoinSideSpec, dim: JoinSideSpec, key_domain: int,
                   dim2: JoinSideSpec | None = None, key_domain2: int = 0, dim_fk2_col: int = 0,
                   method: int = GACE_JOIN_AUTO):
    """dict(card, fact_rows, dim_rows, dim2_rows) of the (chain) join."""
    spec = _capi.gace_join()
    fact.fill(spec.fact)
    dim.fill(spec.dim)
    spec.key_domain = key_domain
    if dim2 is not None:
        dim2.fill(spec.dim2)
        spec.key_domain2 = key_domain2
        spec.dim_fk2_col = dim_fk2_col
        spec.hops = 2
    else:
        spec.hops = 1
    spec.method = method
    out = _capi.gace_join_result()
    check(lib().gace_join_card(ctx, C.byref(spec), C.byref(out)), "gace_join_card")
    return {"card": int(out.card), "fact_rows": int(out.fact_rows), "dim_rows": int(out.dim_rows),
            "dim2_rows": int(out.dim2_rows)}


# ----------------------------------------------------------------- resident samples and sketches

def gace_sample_materialize(ctx, table_id: int, sample):
    """(sample table id, its rows): the rows of a row or block sample of a
    table, every column, in row order, as a new table of the context."""
    out = C.c_uint32()
    rows = C.c_uint64()
    smp = _samples([sample])
    check(lib().gace_sample_materialize(ctx, table_id, smp, C.byref(out), C.byref(rows)), "gace_sample_materialize")
    return int(out.value), int(rows.value)


def gace_resident_configure(ctx, budget_bytes: int, admit_after: int = 0, samples: bool = True,
                            sketches: bool = True) -> None:
    """Turns the resident store of samples and sketches on (budget_bytes > 0)
    or off (0)."""
    flags = (_capi.GACE_RESIDENT_SAMPLES if samples else 0) | (_capi.GACE_RESIDENT_SKETCHES if sketches else 0)
    if budget_bytes and not flags:
        raise ValueError("a resident store keeps samples, sketches or both")
    cfg = _capi.gace_resident_config(int(budget_bytes), int(admit_after), flags)
    check(lib().gace_resident_configure(ctx, C.byref(cfg)), "gace_resident_configure")


def gace_resident_prefetch(ctx, table_id: int, sample) -> None:
    """Materialises a sample into the resident store now."""
    check(lib().gace_resident_prefetch(ctx, table_id, _samples([sample])), "gace_resident_prefetch")


def gace_resident_stats_read(ctx) -> dict:
    st = _capi.gace_resident_stats()
    check(lib().gace_resident_stats_read(ctx, C.byref(st)), "gace_resident_stats_read")
    return {k: int(getattr(st, k)) for k, _ in _capi.gace_resident_stats._fields_}


# ----------------------------------------------------------------- batched form

class ProbeRequest:
    """A probe request of a batch; after the batch, .results / .marginals
    hold what gace_probe_batch would return."""

    def __init__(self, table_id: int, preds, samples, dtypes, marginals: bool = False,
                 batch: TermBatch | None = None):
        self.table_id = table_id
        self.b = batch or TermBatch(preds, dtypes)
        self.smp = _samples(samples)
        self.nsamples = len(samples)
        self.results = np.zeros((len(samples), self.b.npreds), dtype=RESULT_DTYPE)
        self.marginals = np.zeros((len(samples), self.b.nterms), dtype=np.uint64) if marginals else None
        self.req = _capi.gace_request()
        self.fill(self.req)

    def fill(self, r):
        r.kind, r.table_id = _capi.GACE_REQ_PROBE, self.table_id
        r.samples, r.nsamples = C.cast(self.smp, C.POINTER(_capi.gace_sample)), self.nsamples
        r.terms, r.nterms = C.cast(self.b.terms, C.POINTER(_capi.gace_term)), self.b.nterms
        r.in_values, r.nin = C.cast(self.b.in_values, C.POINTER(_capi.gace_scalar)), self.b.nin
        r.preds, r.npreds = C.cast(self.b.preds, C.POINTER(_capi.gace_pred)), self.b.npreds
        r.results = self.results.ctypes.data_as(C.POINTER(_capi.gace_pred_result))
        r.term_marginals = (self.marginals.ctypes.data_as(C.POINTER(C.c_uint64))
                            if self.marginals is not None and self.b.nterms else None)


class NdvRequest:
    """An HLL request of a batch; after the batch, .registers / .estimate."""

    def __init__(self, table_id: int, col: int, p: int, hash_seed: int):
        self.table_id, self.col, self.p, self.seed = table_id, col, p, int(hash_seed) & ((1 << 64) - 1)
        self.registers = np.zeros(1 << p, dtype=np.uint8)
        self._est = C.c_double()
        self.req = _capi.gace_request()
        self.fill(self.req)

    @property
    def estimate(self) -> float:
        return float(self._est.value)

    def fill(self, r):
        r.kind, r.table_id, r.col, r.p, r.hash_seed = _capi.GACE_REQ_NDV, self.table_id, self.col, self.p, self.seed
        r.registers_out = self.registers.ctypes.data_as(C.POINTER(C.c_uint8))
        r.estimate_out = C.pointer(self._est)


class JoinRequest:
    """A join request of a batch; after the batch, .result (as gace_join_card)."""

    def __init__(self, fact: "JoinSideSpec", dim: "JoinSideSpec", key_domain: int, dim2=None,
                 key_domain2: int = 0, dim_fk2_col: int = 0, method: int = GACE_JOIN_AUTO):
        self.sides = (fact, dim, dim2)
        self.spec = _capi.gace_join()
        fact.fill(self.spec.fact)
        dim.fill(self.spec.dim)
        self.spec.key_domain = key_domain
        if dim2 is not None:
            dim2.fill(self.spec.dim2)
            self.spec.key_domain2, self.spec.dim_fk2_col, self.spec.hops = key_domain2, dim_fk2_col, 2
        else:
            self.spec.hops = 1
        self.spec.method = method
        self.out = _capi.gace_join_result()
        self.req = _capi.gace_request()
        self.fill(self.req)

    @property
    def result(self) -> dict:
        o = self.out
        return {"card": int(o.card), "fact_rows": int(o.fact_rows), "dim_rows": int(o.dim_rows),
                "dim2_rows": int(o.dim2_rows)}

    def fill(self, r):
        r.kind = _capi.GACE_REQ_JOIN
        r.join = C.pointer(self.spec)
        r.join_out = C.pointer(self.out)


def _request_array(requests):
    if isinstance(requests, RequestArray):
        return requests.arr
    arr = (_capi.gace_request * max(1, len(requests)))()
    for k, q in enumerate(requests):
        arr[k] = q.req
    return arr


class RequestArray:
    """The C array of a list of request objects, marshalled once and passed
    to gace_run_batch / gace_tune_batch any number of times (every run writes
    the requests' outputs again)."""

    def __init__(self, requests):
        self.requests = list(requests)
        self.arr = _request_array(self.requests)

    def __len__(self):
        return len(self.requests)


def gace_run_batch(ctx, requests, raise_on_error: bool = True):
    """Runs ProbeRequest / NdvRequest / JoinRequest objects (a list or a
    RequestArray) as one batch; returns the per-request statuses (and raises
    on the first failure unless raise_on_error is False)."""
    arr = _request_array(requests)
    n = len(requests)
    st = (C.c_int * max(1, n))()
    rc = lib().gace_run_batch(ctx, arr, n, st)
    if raise_on_error:
        check(rc, "gace_run_batch")
    return [int(st[i]) for i in range(n)]


def gace_tune_batch(ctx, requests) -> None:
    """Tunes the batched form for batches shaped like `requests` (a list or a
    RequestArray); the requests receive their outputs."""
    arr = _request_array(requests)
    check(lib().gace_tune_batch(ctx, arr, len(requests)), "gace_tune_batch")


def gace_tune_save(ctx, path: str) -> None:
    check(lib().gace_tune_save(ctx, path.encode()), "gace_tune_save")


def gace_tune_load(ctx, path: str) -> None:
    check(lib().gace_tune_load(ctx, path.encode()), "gace_tune_load")


# ----------------------------------------------------------------- served form

_SUBMITTED: dict = {}  # (context, ticket) -> request object whose outputs are pending


def gace_serve_start(ctx, arena_bytes: int = 0, max_inflight: int = 0, sketch_cache: int = 0,
                     step_rows: int = 0, chunk_rows: int = 0, always_step: bool = False,
                     probe_cache: int = 0, idle_spin_us: int = 0, fuse_samples: bool = False) -> None:
    flags = (_capi.GACE_SERVE_ALWAYS_STEP if always_step else 0) | \
        (_capi.GACE_SERVE_FUSE_SAMPLES if fuse_samples else 0)
    cfg = _capi.gace_serve_config(arena_bytes, max_inflight, sketch_cache, step_rows, chunk_rows, flags,
                                  probe_cache, idle_spin_us)
    check(lib().gace_serve_start(ctx, C.byref(cfg)), "gace_serve_start")


def gace_serve_stop(ctx) -> None:
    check(lib().gace_serve_stop(ctx), "gace_serve_stop")
    for key in [k for k in _SUBMITTED if k[0] == _ctx_key(ctx)]:
        del _SUBMITTED[key]


def _ctx_key(ctx) -> int:
    return C.cast(ctx, C.c_void_p).value or 0


def gace_submit(ctx, request) -> int:
    """Queues a ProbeRequest / NdvRequest / JoinRequest; returns its ticket.
    The request object receives the outputs once gace_poll reports completion."""
    t = C.c_uint64()
    check(lib().gace_submit(ctx, C.byref(request.req), C.byref(t)), "gace_submit")
    _SUBMITTED[(_ctx_key(ctx), t.value)] = request
    return t.value


def gace_poll(ctx, ticket: int, timeout_us: int = 0) -> bool:
    """True once the request has completed (its outputs are in the request
    object), False while it is pending; raises GaceError if it failed."""
    rc = lib().gace_poll(ctx, ticket, timeout_us)
    if rc == GACE_EPENDING:
        return False
    _SUBMITTED.pop((_ctx_key(ctx), ticket), None)
    check(rc, "gace_poll")
    return True


def gace_serve_replay(ctx, requests, arrival_ns, mode: int = 0):
    """Open-loop replay: request i is submitted at arrival_ns[i] nanoseconds
    after the start (mode 0 served, mode 1 one synchronous call per request).
    Returns (done_ns, statuses) as numpy arrays."""
    n = len(requests)
    arr = _request_array(requests)
    arrival = np.ascontiguousarray(arrival_ns, dtype=np.uint64)
    done = np.zeros(max(1, n), dtype=np.uint64)
    st = np.zeros(max(1, n), dtype=np.int32)
    lib().gace_serve_replay(ctx, arr, n, arrival.ctypes.data_as(C.POINTER(C.c_uint64)), mode,
                            done.ctypes.data_as(C.POINTER(C.c_uint64)), st.ctypes.data_as(C.POINTER(C.c_int)))
    return done[:n], st[:n]


def gace_run_plain_async(ctxs, requests):
    """Request i (a request object or RequestArray entry whose table ids are
    those of ctxs[i % len(ctxs)]) through its synchronous call on that context,
    one host thread per context; returns the per-request statuses."""
    n = len(requests)
    arr = _request_array(requests)
    cs = (C.c_void_p * len(ctxs))(*ctxs)
    st = np.zeros(max(1, n), dtype=np.int32)
    lib().gace_run_plain_async(cs, len(ctxs), arr, n, st.ctypes.data_as(C.POINTER(C.c_int)))
    return [int(x) for x in st[:n]]


def gace_gate_eval(inputs, config=None):
    """Risky Gate trust metrics (Eq. 1-3) of each input, a dict with keys
    ndv_hist, ndv_est, sel_est, sel_probe, pcs (missing keys are NaN: that
    signal is left out).  config: dict of drift_min, sel_err_max, pcs_high,
    pcs_low (missing or 0 = the paper's thresholds).  Returns (flags, drift,
    sel_err) numpy arrays."""
    n = len(inputs)
    arr = (_capi.gace_gate_input * max(1, n))()
    nan = float("nan")
    for i, x in enumerate(inputs):
        arr[i] = _capi.gace_gate_input(*(float(x.get(k, nan)) for k in
                                         ("ndv_hist", "ndv_est", "sel_est", "sel_probe", "pcs")))
    out = (_capi.gace_gate_result * max(1, n))()
    cfg = None
    if config is not None:
        cfg = C.byref(_capi.gace_gate_config(*(float(config.get(k, 0.0)) for k in
                                               ("drift_min", "sel_err_max", "pcs_high", "pcs_low"))))
    check(lib().gace_gate_eval(cfg, arr, n, out), "gace_gate_eval")
    flags = np.array([out[i].flags for i in range(n)], dtype=np.uint32)
    drift = np.array([out[i].drift for i in range(n)], dtype=np.float64)
    sel_err = np.array([out[i].sel_err for i in range(n)], dtype=np.float64)
    return flags, drift, sel_err


def gace_break_even(ctx, nrows: int, npreds: int, nsets: int = 1, hashed_sets: int = 0, nterms: int | None = None,
                    row_bytes: int = 4, resident: bool = True, ops_per_row: float = 0.0,
                    alt_ms: float = 0.0) -> dict:
    """Predicted cost of one probe and whether it beats alt_ms (the
    break-even logic of Section V); see gace_break_even in gace.h."""
    q = _capi.gace_cost_query(int(nrows), int(npreds), int(nsets), int(hashed_sets),
                              int(npreds if nterms is None else nterms), int(row_bytes), 1 if resident else 0,
                              float(ops_per_row), float(alt_ms))
    a = _capi.gace_cost_answer()
    check(lib().gace_break_even(ctx, C.byref(q), C.byref(a)), "gace_break_even")
    return {k: getattr(a, k) for k, _ in _capi.gace_cost_answer._fields_ if k != "reserved"}


def gace_check_wait_limit(ctx, timeout_us: int) -> int:
    """Runs the bounded-wait check kernel; returns its status code
    (GACE_ETIMEDOUT when the wait gave up as it must)."""
    return int(lib().gace_check_wait_limit(ctx, int(timeout_us)))


def gace_calibrate_int(ctx, kind: int = 0, ms: int = 50) -> float:
    """Integer operations per second this GPU retires (kind 0: xor/add lane
    operations; kind 1: 32-bit range tests), timed on the context stream."""
    out = C.c_double()
    check(lib().gace_calibrate_int(ctx, kind, ms, C.byref(out)), "gace_calibrate_int")
    return float(out.value)


def gace_stats_reset(ctx, time_kernels: bool = False) -> None:
    check(lib().gace_stats_reset(ctx, 1 if time_kernels else 0), "gace_stats_reset")


def gace_stats_read(ctx) -> dict:
    """{kernel family: dict(launches, rows, bytes, ops, total_ms)} since the last reset."""
    n = C.c_uint32()
    check(lib().gace_stats_read(ctx, None, 0, C.byref(n)), "gace_stats_read")
    arr = (_capi.gace_kernel_stat * max(1, n.value))()
    check(lib().gace_stats_read(ctx, arr, n.value, C.byref(n)), "gace_stats_read")
    return {arr[i].name.decode(): {"launches": int(arr[i].launches), "rows": int(arr[i].rows),
                                   "bytes": int(arr[i].bytes), "ops": int(arr[i].ops),
                                   "total_ms": float(arr[i].total_ms)} for i in range(n.value)}


def gace_last_error() -> str:
    return lib().gace_last_error().decode()


def gace_status_string(s: int) -> str:
    return lib().gace_status_string(s).decode()


__all__ = [n for n in dir() if n.startswith(("gace_", "GACE_"))] + [
    "GaceError", "JoinRequest", "JoinSideSpec", "NdvRequest", "ProbeRequest", "RESULT_DTYPE", "RequestArray",
    "TermBatch",
    "check", "lib"]
