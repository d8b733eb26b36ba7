"""Failure detection on the GPU without a fault: a device-side wait that
nothing completes gives up at its limit, the kernel reports the timeout
status, and the context keeps working afterwards."""
import time

import pytest
import torch

from workloads import FULL, I32, RANGE, Sample, Term

pytestmark = pytest.mark.gpu


def test_device_wait_gives_up_and_context_stays_usable(g, gctx, cuda):
    t0 = time.perf_counter()
    st = g.gace_check_wait_limit(gctx, 2000)  # 2 ms
    dt = time.perf_counter() - t0
    assert st == g.GACE_ETIMEDOUT
    assert 0.002 <= dt < 5.0
    # the context (and its stream) still work
    col = torch.arange(100_000, dtype=torch.int32, device=cuda)
    tid = g.gace_load_columns(gctx, [col], borrow=True)
    try:
        res, _ = g.gace_probe_batch(gctx, tid, [[Term(0, RANGE, 0, 500)]], [Sample(FULL)], [I32])
        assert int(res["match"][0, 0]) == 500
    finally:
        g.gace_unload(gctx, tid)
    assert g.gace_check_wait_limit(gctx, 0) == g.GACE_EINVAL
