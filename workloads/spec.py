"""Plain descriptions of probes: terms, predicates and sample specifications.

These are data only -- no arithmetic of the method lives here.  Both the CPU
oracle wrapper and the library binding translate the same descriptions into
their own structures, so the two sides see identical inputs.
"""
from __future__ import annotations

from dataclasses import dataclass, field

# column element types
I32, I64, F32 = 0, 1, 2
# term operators
EQ, RANGE, IN = 0, 1, 2
# sample kinds
FULL, ROWS, BLOCKS = 0, 1, 2

DTYPE_NAMES = {I32: "int32", I64: "int64", F32: "float32"}


@dataclass(frozen=True)
class Term:
    """One candidate condition on a column.

    EQ: x == a.  RANGE: a <= x < b (half-open).  IN: x in values.
    Integer columns take int constants, float columns float constants.
    """

    col: int
    op: int
    a: float | int = 0
    b: float | int = 0
    values: tuple = ()


@dataclass(frozen=True)
class Sample:
    """Which rows a probe counts over: all of them, a seeded Bernoulli sample
    of rows, or a seeded Bernoulli sample of fixed-size row blocks."""

    kind: int = FULL
    rate: float = 1.0
    seed: int = 0
    block_rows: int = 4096


@dataclass
class Table:
    """A synthetic columnar table.  columns are torch tensors (any device)."""

    name: str
    columns: list
    dtypes: list
    domains: list = field(default_factory=list)

    @property
    def nrows(self) -> int:
        return int(self.columns[0].shape[0]) if self.columns else 0


@dataclass
class JoinSide:
    """A table, its join-key column and a conjunctive filter (list of Terms)."""

    table: Table
    key_col: int
    terms: list = field(default_factory=list)
