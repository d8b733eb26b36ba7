"""Seeded synthetic inputs for the probe path, shared by the oracle and the GPU
library as plain data (tables, predicate batches, sample specifications)."""
from .gen import (copula_zipf_pair, make_batched, make_join, make_plain_small, make_predicates,
                  make_skew_corr, normal_column, uniform_int_column, zipf_column)
from .spec import (BLOCKS, EQ, F32, FULL, I32, I64, IN, RANGE, ROWS, JoinSide, Sample,
                   Table, Term)

__all__ = [
    "BLOCKS", "EQ", "F32", "FULL", "I32", "I64", "IN", "RANGE", "ROWS",
    "JoinSide", "Sample", "Table", "Term",
    "copula_zipf_pair", "make_batched", "make_join", "make_plain_small", "make_predicates",
    "make_skew_corr", "normal_column", "uniform_int_column", "zipf_column",
]
