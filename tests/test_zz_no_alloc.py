"""The no-allocation HyperLogLog entry point (gace_ndv_noalloc) against the
CPU oracle and against the context-based entry point (gace_ndv).

gace_ndv_noalloc exists for callers that cannot allocate device memory (a
planning hook that must not trigger cudaMalloc's device-wide synchronisation,
or a process whose device memory belongs to another allocator).  It keeps its
scratch in a fixed array inside the library that every call reuses, so two
calls in a row must each clear it and each give the oracle's registers.  After
one warm-up call (which may load the library's module on the device), a call
must leave the device's free memory unchanged.  This file is collected last
so that a failure here leaves every other test already run."""
import numpy as np
import pytest
import torch

from parity import close
from workloads import F32, I32, I64

pytestmark = pytest.mark.gpu


def _columns(cuda):
    g = torch.Generator(device=cuda)
    g.manual_seed(99)
    a = torch.randint(-2**31, 2**31, (3_000_017,), generator=g, device=cuda, dtype=torch.int64).to(torch.int32)
    b = torch.randint(0, 50_000, (1_234_567,), generator=g, device=cuda, dtype=torch.int64)
    c = torch.randn(777_777, generator=g, device=cuda, dtype=torch.float32)
    return [a, b, c], [I32, I64, F32]


def test_two_calls_in_a_row_match_the_oracle(g, orc, gctx, cuda):
    cols, dtypes = _columns(cuda)
    host = [c.cpu().numpy() for c in cols]
    cases = [(0, 16, 42), (1, 12, 7), (2, 14, 3), (0, 16, 42)]
    tids = [g.gace_load_columns(gctx, [c], borrow=True) for c in cols]
    try:
        for col, p, seed in cases:
            regs, est = g.gace_ndv_noalloc(cols[col], p, seed)
            ref = orc.hll_registers(host[col], dtypes[col], p, seed)
            bad = np.nonzero(regs != ref)[0]
            assert len(bad) == 0, (col, p, len(bad), bad[:5])
            assert close(est, orc.hll_estimate(ref, p)), (est, orc.hll_estimate(ref, p))
            # the context-based entry point: the same registers, the same double
            ctx_regs, ctx_est = g.gace_ndv(gctx, tids[col], 0, p, seed)
            assert np.array_equal(regs, ctx_regs) and est == ctx_est
            assert regs.any()
    finally:
        for t in tids:
            g.gace_unload(gctx, t)


def test_a_call_leaves_free_device_memory_unchanged(g, orc, cuda):
    cols, dtypes = _columns(cuda)
    g.gace_ndv_noalloc(cols[0], 16, 5)  # warm-up: the module is loaded on this device
    side = torch.cuda.Stream(device=cuda)
    torch.cuda.synchronize(cuda)
    free_before, _ = torch.cuda.mem_get_info(cuda)
    regs, _ = g.gace_ndv_noalloc(cols[2], 14, 11, stream=side)
    free_after, _ = torch.cuda.mem_get_info(cuda)
    assert free_after == free_before, (free_before, free_after)
    assert np.array_equal(regs, orc.hll_registers(cols[2].cpu().numpy(), F32, 14, 11))


def test_empty_column_and_limit(g, cuda):
    empty = torch.zeros(0, dtype=torch.int32, device=cuda)
    regs, est = g.gace_ndv_noalloc(empty, 10, 1)
    assert not regs.any() and est == 0.0
    col = torch.arange(1000, dtype=torch.int32, device=cuda)
    with pytest.raises(g.GaceError) as e:
        g.gace_ndv_noalloc(col, 17, 1)
    assert e.value.status == 1 and "16" in e.value.message
