"""ctypes declarations of the C ABI in include/gace.h (marshalling only).

The library is built in-tree (``paper_2512_19750_gb300/libgace.so``).  If it
is missing the import of this module fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgace.so")

GACE_OK, GACE_EINVAL, GACE_ENOMEM, GACE_EBUSY, GACE_EPENDING = 0, 1, 2, 3, 4
GACE_ETIMEDOUT, GACE_ENOTFOUND, GACE_EOVERFLOW, GACE_ECUDA = 5, 6, 7, 8
GACE_I32, GACE_I64, GACE_F32 = 0, 1, 2
GACE_EQ, GACE_RANGE, GACE_IN = 0, 1, 2
GACE_FULL, GACE_ROWS, GACE_BLOCKS = 0, 1, 2
GACE_COPY, GACE_BORROW, GACE_COPY_ON_FIRST_PROBE = 0, 1, 2
GACE_JOIN_AUTO, GACE_JOIN_HIST_DOT, GACE_JOIN_GATHER = 0, 1, 2
GACE_REQ_PROBE, GACE_REQ_NDV, GACE_REQ_JOIN = 0, 1, 2


class gace_scalar(C.Union):
    _fields_ = [("i", C.c_int64), ("f", C.c_double)]


class gace_config(C.Structure):
    _fields_ = [("device", C.c_int32), ("wait_timeout_ms", C.c_uint32),
                ("hbm_budget_bytes", C.c_uint64), ("stream", C.c_void_p), ("max_ctas", C.c_uint32),
                ("rank_min_rows", C.c_uint32), ("rank_search", C.c_uint32)]


class gace_column(C.Structure):
    _fields_ = [("dtype", C.c_int32), ("on_device", C.c_int32), ("data", C.c_void_p)]


class gace_term(C.Structure):
    _fields_ = [("col", C.c_uint32), ("op", C.c_uint32), ("a", gace_scalar), ("b", gace_scalar),
                ("in_off", C.c_uint32), ("in_len", C.c_uint32)]


class gace_pred(C.Structure):
    _fields_ = [("term_off", C.c_uint32), ("term_cnt", C.c_uint32)]


class gace_sample(C.Structure):
    _fields_ = [("kind", C.c_uint32), ("block_rows", C.c_uint32), ("rate", C.c_double),
                ("seed", C.c_uint64)]


class gace_pred_result(C.Structure):
    _fields_ = [("match", C.c_uint64), ("sample_rows", C.c_uint64), ("sel", C.c_double),
                ("pcs", C.c_double)]


class gace_join_side(C.Structure):
    _fields_ = [("table_id", C.c_uint32), ("key_col", C.c_uint32),
                ("terms", C.POINTER(gace_term)), ("nterms", C.c_uint32), ("nin", C.c_uint32),
                ("in_values", C.POINTER(gace_scalar))]


class gace_join(C.Structure):
    _fields_ = [("fact", gace_join_side), ("dim", gace_join_side), ("key_domain", C.c_uint64),
                ("dim2", gace_join_side), ("key_domain2", C.c_uint64),
                ("dim_fk2_col", C.c_uint32), ("hops", C.c_uint32), ("method", C.c_uint32),
                ("reserved", C.c_uint32)]


class gace_join_result(C.Structure):
    _fields_ = [("card", C.c_int64), ("fact_rows", C.c_uint64), ("dim_rows", C.c_uint64),
                ("dim2_rows", C.c_uint64)]


class gace_request(C.Structure):
    _fields_ = [("kind", C.c_uint32), ("table_id", C.c_uint32),
                ("samples", C.POINTER(gace_sample)), ("nsamples", C.c_uint32),
                ("nterms", C.c_uint32), ("terms", C.POINTER(gace_term)),
                ("in_values", C.POINTER(gace_scalar)), ("nin", C.c_uint32), ("npreds", C.c_uint32),
                ("preds", C.POINTER(gace_pred)), ("results", C.POINTER(gace_pred_result)),
                ("term_marginals", C.POINTER(C.c_uint64)), ("col", C.c_uint32), ("p", C.c_uint32),
                ("hash_seed", C.c_uint64), ("registers_out", C.POINTER(C.c_uint8)),
                ("estimate_out", C.POINTER(C.c_double)), ("join", C.POINTER(gace_join)),
                ("join_out", C.POINTER(gace_join_result))]


GACE_SERVE_ALWAYS_STEP = 1
GACE_SERVE_FUSE_SAMPLES = 2


class gace_serve_config(C.Structure):
    _fields_ = [("arena_bytes", C.c_uint64), ("max_inflight", C.c_uint32), ("sketch_cache", C.c_int32),
                ("step_rows", C.c_uint64), ("chunk_rows", C.c_uint64), ("flags", C.c_uint32),
                ("probe_cache", C.c_int32), ("idle_spin_us", C.c_uint32)]


class gace_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("launches", C.c_uint64), ("rows", C.c_uint64),
                ("bytes", C.c_uint64), ("ops", C.c_uint64), ("total_ms", C.c_double)]


class gace_gate_config(C.Structure):
    _fields_ = [("drift_min", C.c_double), ("sel_err_max", C.c_double), ("pcs_high", C.c_double),
                ("pcs_low", C.c_double)]


class gace_gate_input(C.Structure):
    _fields_ = [("ndv_hist", C.c_double), ("ndv_est", C.c_double), ("sel_est", C.c_double),
                ("sel_probe", C.c_double), ("pcs", C.c_double)]


class gace_gate_result(C.Structure):
    _fields_ = [("flags", C.c_uint32), ("reserved", C.c_uint32), ("drift", C.c_double), ("sel_err", C.c_double)]


class gace_cost_query(C.Structure):
    _fields_ = [("nrows", C.c_uint64), ("npreds", C.c_uint32), ("nsets", C.c_uint32), ("hashed_sets", C.c_uint32),
                ("nterms", C.c_uint32), ("row_bytes", C.c_uint32), ("resident", C.c_uint32),
                ("ops_per_row", C.c_double), ("alt_ms", C.c_double)]


class gace_cost_answer(C.Structure):
    _fields_ = [("total_ms", C.c_double), ("kernel_ms", C.c_double), ("transfer_ms", C.c_double),
                ("call_ms", C.c_double), ("hbm_rate", C.c_double), ("ops_rate", C.c_double),
                ("h2d_rate", C.c_double), ("hash_ns", C.c_double), ("narrow", C.c_uint32),
                ("offload", C.c_uint32), ("measured", C.c_uint32), ("reserved", C.c_uint32)]


GACE_RISK_DRIFT, GACE_RISK_SELECTIVITY, GACE_RISK_CORRELATION = 1, 2, 4
GACE_RESIDENT_SAMPLES, GACE_RESIDENT_SKETCHES = 1, 2


class gace_resident_config(C.Structure):
    _fields_ = [("budget_bytes", C.c_uint64), ("admit_after", C.c_uint32), ("flags", C.c_uint32)]


class gace_resident_stats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in (
        "budget_bytes", "used_bytes", "samples", "sketches", "sample_hits", "sample_misses", "admitted",
        "refused", "evicted", "sketch_hits", "sketch_misses", "sketch_evicted")]

ctx_p = C.c_void_p

# name -> (restype, argtypes); every function declared in include/gace.h
PROTOTYPES = {
    "gace_create": (C.c_int, [C.POINTER(ctx_p), C.POINTER(gace_config)]),
    "gace_destroy": (C.c_int, [ctx_p]),
    "gace_load_columns": (C.c_int, [ctx_p, C.c_uint64, C.c_uint32, C.POINTER(gace_column),
                                    C.c_uint32, C.POINTER(C.c_uint32)]),
    "gace_unload": (C.c_int, [ctx_p, C.c_uint32]),
    "gace_probe_batch": (C.c_int, [ctx_p, C.c_uint32, C.POINTER(gace_sample), C.c_uint32,
                                   C.POINTER(gace_term), C.c_uint32, C.POINTER(gace_scalar),
                                   C.c_uint32, C.POINTER(gace_pred), C.c_uint32,
                                   C.POINTER(gace_pred_result), C.POINTER(C.c_uint64)]),
    "gace_ndv": (C.c_int, [ctx_p, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint64,
                           C.POINTER(C.c_uint8), C.POINTER(C.c_double)]),
    "gace_join_card": (C.c_int, [ctx_p, C.POINTER(gace_join), C.POINTER(gace_join_result)]),
    "gace_ndv_noalloc": (C.c_int, [C.c_void_p, C.c_int32, C.c_uint64, C.c_uint32, C.c_uint64,
                                   C.c_void_p, C.POINTER(C.c_uint8), C.POINTER(C.c_double)]),
    "gace_sample_materialize": (C.c_int, [ctx_p, C.c_uint32, C.POINTER(gace_sample), C.POINTER(C.c_uint32),
                                          C.POINTER(C.c_uint64)]),
    "gace_resident_configure": (C.c_int, [ctx_p, C.POINTER(gace_resident_config)]),
    "gace_resident_prefetch": (C.c_int, [ctx_p, C.c_uint32, C.POINTER(gace_sample)]),
    "gace_resident_stats_read": (C.c_int, [ctx_p, C.POINTER(gace_resident_stats)]),
    "gace_run_batch": (C.c_int, [ctx_p, C.POINTER(gace_request), C.c_uint32, C.POINTER(C.c_int)]),
    "gace_tune_batch": (C.c_int, [ctx_p, C.POINTER(gace_request), C.c_uint32]),
    "gace_tune_save": (C.c_int, [ctx_p, C.c_char_p]),
    "gace_tune_load": (C.c_int, [ctx_p, C.c_char_p]),
    "gace_serve_start": (C.c_int, [ctx_p, C.POINTER(gace_serve_config)]),
    "gace_serve_stop": (C.c_int, [ctx_p]),
    "gace_submit": (C.c_int, [ctx_p, C.POINTER(gace_request), C.POINTER(C.c_uint64)]),
    "gace_poll": (C.c_int, [ctx_p, C.c_uint64, C.c_uint64]),
    "gace_serve_replay": (C.c_int, [ctx_p, C.POINTER(gace_request), C.c_uint32, C.POINTER(C.c_uint64),
                                    C.c_uint32, C.POINTER(C.c_uint64), C.POINTER(C.c_int)]),
    "gace_run_plain_async": (C.c_int, [C.POINTER(ctx_p), C.c_uint32, C.POINTER(gace_request), C.c_uint32,
                                       C.POINTER(C.c_int)]),
    "gace_gate_eval": (C.c_int, [C.POINTER(gace_gate_config), C.POINTER(gace_gate_input), C.c_uint32,
                                 C.POINTER(gace_gate_result)]),
    "gace_break_even": (C.c_int, [ctx_p, C.POINTER(gace_cost_query), C.POINTER(gace_cost_answer)]),
    "gace_check_wait_limit": (C.c_int, [ctx_p, C.c_uint32]),
    "gace_calibrate_int": (C.c_int, [ctx_p, C.c_uint32, C.c_uint32, C.POINTER(C.c_double)]),
    "gace_stats_reset": (C.c_int, [ctx_p, C.c_uint32]),
    "gace_stats_read": (C.c_int, [ctx_p, C.POINTER(gace_kernel_stat), C.c_uint32,
                                  C.POINTER(C.c_uint32)]),
    "gace_last_error": (C.c_char_p, []),
    "gace_status_string": (C.c_char_p, [C.c_int]),
    "gace_abi_version": (C.c_uint32, []),
}

_lib = None


def lib():
    """The loaded libgace.so with prototypes attached (raises if not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in PROTOTYPES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class GaceError(RuntimeError):
    def __init__(self, status: int, where: str):
        L = lib()
        self.status = status
        self.name = L.gace_status_string(status).decode()
        self.message = L.gace_last_error().decode()
        super().__init__(f"{where}: {self.name}: {self.message}")


def check(status: int, where: str) -> None:
    if status != GACE_OK:
        raise GaceError(status, where)
