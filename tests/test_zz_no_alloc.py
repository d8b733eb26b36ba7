"""The no-allocation HyperLogLog entry point (gace_ndv_noalloc) against the
context-based one (gace_ndv).

gace_ndv_noalloc exists for callers that cannot allocate device memory (a
planning hook that must not trigger cudaMalloc's device-wide synchronisation,
or a process whose device memory belongs to another allocator).  It keeps its
scratch in a fixed array inside the library that every call reuses, so two
calls in a row must each clear it and each give the context-based result.
This file is collected last so that a failure here leaves every other test
already run."""
import numpy as np
import pytest
import torch

from parity import close

pytestmark = pytest.mark.gpu


def _columns(cuda):
    g = torch.Generator(device=cuda)
    g.manual_seed(99)
    a = torch.randint(-2**31, 2**31, (3_000_017,), generator=g, device=cuda, dtype=torch.int64).to(torch.int32)
    b = torch.randint(0, 50_000, (1_234_567,), generator=g, device=cuda, dtype=torch.int64)
    c = torch.randn(777_777, generator=g, device=cuda, dtype=torch.float32)
    return [a, b, c]


def test_two_calls_in_a_row_match_gace_ndv(g, gctx, cuda):
    cols = _columns(cuda)
    cases = [(0, 16, 42), (1, 12, 7), (2, 14, 3), (0, 16, 42)]
    tids = [g.gace_load_columns(gctx, [c], borrow=True) for c in cols]
    try:
        for col, p, seed in cases:
            regs, est = g.gace_ndv_noalloc(cols[col], p, seed)
            ref_regs, ref_est = g.gace_ndv(gctx, tids[col], 0, p, seed)
            assert np.array_equal(regs, ref_regs), (col, p)
            assert close(est, ref_est), (est, ref_est)
            assert regs.any()
    finally:
        for t in tids:
            g.gace_unload(gctx, t)


def test_empty_column_and_limit(g, cuda):
    empty = torch.zeros(0, dtype=torch.int32, device=cuda)
    regs, est = g.gace_ndv_noalloc(empty, 10, 1)
    assert not regs.any() and est == 0.0
    col = torch.arange(1000, dtype=torch.int32, device=cuda)
    with pytest.raises(g.GaceError) as e:
        g.gace_ndv_noalloc(col, 17, 1)
    assert e.value.status == 1 and "16" in e.value.message
