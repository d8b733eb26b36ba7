"""GPU parity of HyperLogLog (K4): registers bit-exact against the oracle for
every column type, register count and odd size; estimates within 1e-12."""
import numpy as np
import pytest
import torch

from parity import close
from workloads import F32, I32, I64, make_skew_corr

pytestmark = pytest.mark.gpu


def _check(g, orc, ctx, tid, col_host, dtype, col, p, seed):
    regs, est = g.gace_ndv(ctx, tid, col, p, seed)
    ref = orc.hll_registers(col_host, dtype, p, seed)
    bad = np.nonzero(regs != ref)[0]
    assert len(bad) == 0, f"p={p}: {len(bad)} registers differ, first {bad[:5]}: {regs[bad[:5]]} vs {ref[bad[:5]]}"
    assert close(est, orc.hll_estimate(ref, p))
    return regs, est


@pytest.mark.parametrize("p", [4, 5, 6, 7, 10, 12, 14, 16, 17, 18])
def test_registers_every_precision(g, gctx, orc, cuda, p):
    t = make_skew_corr(n=150_001, seed=40 + p, device=cuda, domain=200_000)
    tid = g.gace_load_columns(gctx, t.columns)
    try:
        for c in (0, 4, 6):
            _check(g, orc, gctx, tid, t.columns[c].cpu(), t.dtypes[c], c, p, 42 + c)
    finally:
        g.gace_unload(gctx, tid)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 5, 31, 1000, 4097, 100_003])
def test_registers_odd_sizes(g, gctx, orc, cuda, n):
    rng = np.random.default_rng(n)
    cols = [rng.integers(-2**31, 2**31, n, dtype=np.int64).astype(np.int32),
            rng.integers(-2**62, 2**62, n, dtype=np.int64),
            rng.standard_normal(n).astype(np.float32)]
    tid = g.gace_load_columns(gctx, cols)
    try:
        for c, dt in enumerate((I32, I64, F32)):
            regs, est = _check(g, orc, gctx, tid, cols[c], dt, c, 12, 7)
            if n == 0:
                assert not regs.any() and est == 0.0
    finally:
        g.gace_unload(gctx, tid)


def test_float_canonical_keys(g, gctx, orc):
    vals = np.array([0.0, -0.0, np.nan, -np.nan, np.inf, -np.inf, 1.0, -1.0], dtype=np.float32)
    nan2 = np.frombuffer(np.array([0x7FC00001, 0xFFC12345], dtype=np.uint32).tobytes(), dtype=np.float32)
    col = np.concatenate([vals, nan2])
    tid = g.gace_load_columns(gctx, [col])
    try:
        regs, _ = _check(g, orc, gctx, tid, col, F32, 0, 10, 3)
        assert np.count_nonzero(regs) <= 6  # +-0 one key, every NaN one key
    finally:
        g.gace_unload(gctx, tid)


def test_misaligned_column(g, gctx, orc, cuda):
    base = torch.arange(0, 50_001, dtype=torch.int64, device=cuda) * 7919 % 100_003
    buf = torch.empty(base.numel() + 1, dtype=torch.int64, device=cuda)
    buf[1:] = base
    col = buf[1:]
    assert col.data_ptr() % 16 != 0
    tid = g.gace_load_columns(gctx, [col], borrow=True)
    try:
        _check(g, orc, gctx, tid, base.cpu(), I64, 0, 14, 11)
    finally:
        g.gace_unload(gctx, tid)


def test_errors(g, gctx, cuda):
    tid = g.gace_load_columns(gctx, [torch.zeros(10, dtype=torch.int32, device=cuda)])
    try:
        for p in (3, 19):
            with pytest.raises(g.GaceError) as e:
                g.gace_ndv(gctx, tid, 0, p, 1)
            assert e.value.status == 1
        with pytest.raises(g.GaceError):
            g.gace_ndv(gctx, tid, 1, 12, 1)
    finally:
        g.gace_unload(gctx, tid)
