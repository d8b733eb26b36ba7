"""The library's Risky Gate trust metrics (host code, no GPU) against the
oracle's Eq. 1-3 on random and boundary inputs, and their argument errors."""
import math

import numpy as np
import pytest


def _inputs(rng, n):
    nan = float("nan")
    out = []
    for _ in range(n):
        x = {}
        if rng.random() < 0.8:
            x["ndv_hist"] = float(rng.choice([0.0, -1.0, float("inf"), nan, 1000.0, float(rng.integers(1, 10**7))]))
            x["ndv_est"] = float(rng.choice([nan, 1250.0, 750.0, float(rng.integers(0, 2 * 10**7))]))
        if rng.random() < 0.8:
            x["sel_est"] = float(rng.choice([nan, 0.5, rng.random()]))
            x["sel_probe"] = float(rng.choice([0.51, 0.49, 0.515625, rng.random()]))
        if rng.random() < 0.8:
            x["pcs"] = float(rng.choice([nan, 0.7, 1.6, 0.0, float("inf"), rng.random() * 3]))
        out.append(x)
    return out


@pytest.mark.parametrize("config", [None, {"drift_min": 0.1, "sel_err_max": 0.05, "pcs_high": 2.0, "pcs_low": 0.5},
                                    {"pcs_high": 1.2}])
def test_gate_equals_oracle(g, orc, config):
    rng = np.random.default_rng(11)
    xs = _inputs(rng, 3000)
    flags, drift, sel_err = g.gace_gate_eval(xs, config)
    kw = {}
    if config:
        kw = {k: v for k, v in config.items() if v}
    for i, x in enumerate(xs):
        f, d, e = orc.gate(**x, **kw)
        assert flags[i] == f, (x, flags[i], f)
        assert (math.isnan(d) and math.isnan(drift[i])) or d == drift[i], (x, d, drift[i])
        assert (math.isnan(e) and math.isnan(sel_err[i])) or e == sel_err[i], (x, e, sel_err[i])


def test_gate_argument_errors(g):
    for bad in ({"drift_min": -0.1}, {"pcs_high": float("nan")}, {"sel_err_max": float("inf")},
                {"pcs_high": 0.5, "pcs_low": 0.6}):
        with pytest.raises(g.GaceError) as e:
            g.gace_gate_eval([{"pcs": 1.0}], bad)
        assert e.value.status == g.GACE_EINVAL
    assert len(g.gace_gate_eval([], None)[0]) == 0
