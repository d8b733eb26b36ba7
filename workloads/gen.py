"""Seeded synthetic tables and predicate batches for the probe workloads.

Shapes and distributions follow the evaluation setting of the paper (a
synthetic table of 10^6 rows with a Zipf s = 1.2 skewed column and
multi-column conjunctive filters, Section IV-A) scaled to the five workloads
the probe is measured on.  All randomness comes from torch generators seeded
explicitly, so a (seed, device type) pair always yields the same table.
Nothing here computes a probe result: the oracle and the GPU library both
consume these arrays as inputs.

Zipf(s, D): value v in [0, D) with P(v) proportional to (v + 1)^-s, sampled by
inverse CDF (a float64 cumulative table and a sorted search).
Correlated pairs: Gaussian copula with latent correlation rho -- a shared
standard normal L and z_c = sqrt(rho) L + sqrt(1 - rho) e_c, mapped through
the normal CDF and the Zipf inverse CDF.  rho is the latent (Pearson)
correlation of z, not of the Zipf values.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .spec import EQ, F32, I32, I64, IN, RANGE, Table, Term

_CHUNK = 1 << 25


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=torch.device(device))
    g.manual_seed(int(seed))
    return g


_cdf_cache: dict = {}


def zipf_cdf(s: float, domain: int, device) -> torch.Tensor:
    key = (float(s), int(domain), str(torch.device(device)))
    if key not in _cdf_cache:
        k = torch.arange(1, domain + 1, dtype=torch.float64, device=device)
        w = k.pow(-float(s))
        cdf = torch.cumsum(w, 0)
        cdf /= cdf[-1].clone()
        _cdf_cache[key] = cdf
    return _cdf_cache[key]


def zipf_from_uniform(u: torch.Tensor, s: float, domain: int) -> torch.Tensor:
    cdf = zipf_cdf(s, domain, u.device)
    v = torch.searchsorted(cdf, u, right=True)
    return v.clamp_(max=domain - 1)


def _fill(n: int, dtype, device, fn) -> torch.Tensor:
    out = torch.empty(n, dtype=dtype, device=device)
    for lo in range(0, n, _CHUNK):
        hi = min(n, lo + _CHUNK)
        out[lo:hi] = fn(hi - lo)
    return out


def zipf_column(n, s, domain, g, device, dtype=torch.int32) -> torch.Tensor:
    return _fill(n, dtype, device,
                 lambda m: zipf_from_uniform(
                     torch.rand(m, generator=g, dtype=torch.float64, device=device), s, domain))


def uniform_int_column(n, lo, hi, g, device, dtype=torch.int32) -> torch.Tensor:
    return _fill(n, dtype, device,
                 lambda m: torch.randint(lo, hi, (m,), generator=g, device=device, dtype=torch.int64))


def normal_column(n, g, device) -> torch.Tensor:
    return _fill(n, torch.float32, device,
                 lambda m: torch.randn(m, generator=g, device=device, dtype=torch.float32))


def copula_zipf_pair(n, rho, s, domain, g, device, dtype=torch.int32):
    a = torch.empty(n, dtype=dtype, device=device)
    b = torch.empty(n, dtype=dtype, device=device)
    sr, sn = math.sqrt(rho), math.sqrt(1.0 - rho)
    for lo in range(0, n, _CHUNK):
        hi = min(n, lo + _CHUNK)
        m = hi - lo
        latent = torch.randn(m, generator=g, device=device, dtype=torch.float64)
        e1 = torch.randn(m, generator=g, device=device, dtype=torch.float64)
        e2 = torch.randn(m, generator=g, device=device, dtype=torch.float64)
        u1 = torch.special.ndtr(sr * latent + sn * e1).clamp_(max=1.0 - 2.0 ** -53)
        u2 = torch.special.ndtr(sr * latent + sn * e2).clamp_(max=1.0 - 2.0 ** -53)
        a[lo:hi] = zipf_from_uniform(u1, s, domain)
        b[lo:hi] = zipf_from_uniform(u2, s, domain)
    return a, b


# ----------------------------------------------------------------- workloads

def make_plain_small(n: int = 1_000_000, seed: int = 1001, device="cpu") -> Table:
    """Plain-probe table: c0 uniform on [0, 1e6), c1 Zipf(1.1) over 10^4 values,
    c2 = 7 * c1 + uniform noise on [0, 50) (correlated with c1), c3 uniform on
    [0, 100); all int32."""
    g = _gen(seed, device)
    c0 = uniform_int_column(n, 0, 1_000_000, g, device)
    c1 = zipf_column(n, 1.1, 10_000, g, device)
    noise = uniform_int_column(n, 0, 50, g, device)
    c2 = (c1 * 7 + noise).to(torch.int32)
    c3 = uniform_int_column(n, 0, 100, g, device)
    return Table("plain_small", [c0, c1, c2, c3], [I32] * 4,
                 [1_000_000, 10_000, 70_000, 100])


def make_skew_corr(n: int = 100_000_000, seed: int = 1002, device="cpu",
                   domain: int = 1_000_000) -> Table:
    """Skew + correlation table: c0..c3 int32 Zipf(1.2), c4..c5 int64
    Zipf(1.2), all over `domain` values; c6..c7 float32 N(0, 1).  Pairs
    (c0, c1) and (c4, c5) share a latent normal with rho = 0.9."""
    g = _gen(seed, device)
    c0, c1 = copula_zipf_pair(n, 0.9, 1.2, domain, g, device, torch.int32)
    c2 = zipf_column(n, 1.2, domain, g, device, torch.int32)
    c3 = zipf_column(n, 1.2, domain, g, device, torch.int32)
    c4, c5 = copula_zipf_pair(n, 0.9, 1.2, domain, g, device, torch.int64)
    c6 = normal_column(n, g, device)
    c7 = normal_column(n, g, device)
    return Table("skew_corr", [c0, c1, c2, c3, c4, c5, c6, c7],
                 [I32, I32, I32, I32, I64, I64, F32, F32],
                 [domain] * 6 + [8.0, 8.0])


def make_join(n_fact: int = 500_000_000, n_dim: int = 10_000_000, n_dim2: int = 1_000_000,
              seed: int = 1003, device="cpu", fk_s: float = 1.0):
    """Join tables.  Fact: fk int32 Zipf(1.0) over the n_dim keys, f1 and f2
    uniform on [0, 1000).  Dim: key = seeded permutation of [0, n_dim), g1 and
    g2 uniform on [0, 1000), fk2 uniform on [0, n_dim2) (the chain's foreign
    key).  Dim2: key = permutation of [0, n_dim2), h1, h2 uniform [0, 1000)."""
    g = _gen(seed, device)
    fact = Table("fact", [zipf_column(n_fact, fk_s, n_dim, g, device),
                          uniform_int_column(n_fact, 0, 1000, g, device),
                          uniform_int_column(n_fact, 0, 1000, g, device)],
                 [I32] * 3, [n_dim, 1000, 1000])
    dkey = torch.randperm(n_dim, generator=g, device=device).to(torch.int32)
    dim = Table("dim", [dkey,
                        uniform_int_column(n_dim, 0, 1000, g, device),
                        uniform_int_column(n_dim, 0, 1000, g, device),
                        uniform_int_column(n_dim, 0, n_dim2, g, device)],
                [I32] * 4, [n_dim, 1000, 1000, n_dim2])
    d2key = torch.randperm(n_dim2, generator=g, device=device).to(torch.int32)
    dim2 = Table("dim2", [d2key,
                          uniform_int_column(n_dim2, 0, 1000, g, device),
                          uniform_int_column(n_dim2, 0, 1000, g, device)],
                 [I32] * 3, [n_dim2, 1000, 1000])
    return fact, dim, dim2


# ----------------------------------------------------------------- predicates

def _row_values(col: torch.Tensor, rows: np.ndarray):
    idx = torch.as_tensor(rows, dtype=torch.int64, device=col.device)
    vals = col[idx].cpu()
    return vals.tolist()


def make_predicates(table: Table, npreds: int, min_terms: int, max_terms: int,
                    seed: int, in_len: int = 8):
    """Seeded conjunctive predicates: each has k distinct columns (k uniform in
    [min_terms, max_terms]); integer columns get EQ / RANGE / IN with equal
    probability, float columns RANGE only.  EQ takes the value of a random
    row; RANGE is [x, x + w) with x from a random row and w log-uniform over
    the column's domain; IN lists the values of in_len random rows."""
    rng = np.random.default_rng(seed)
    n = table.nrows
    ncols = len(table.columns)
    preds = []
    plan = []
    for _ in range(npreds):
        k = int(rng.integers(min_terms, max_terms + 1))
        k = min(k, ncols)
        cols = rng.choice(ncols, size=k, replace=False)
        terms = []
        for c in cols:
            c = int(c)
            op = RANGE if table.dtypes[c] == F32 else int(rng.integers(0, 3))
            nrow = in_len if op == IN else 1
            rows = rng.integers(0, max(n, 1), size=nrow)
            width = float(np.exp(rng.uniform(0.0, math.log(max(2.0, table.domains[c])))))
            if table.dtypes[c] == F32:
                width = float(np.exp(rng.uniform(math.log(1e-3), math.log(8.0))))
            terms.append((c, op, rows, width))
        plan.append(terms)
    # fetch all needed row values column by column (few device round trips)
    need = {}
    for terms in plan:
        for c, op, rows, width in terms:
            need.setdefault(c, []).append(rows)
    fetched = {}
    for c, lists in need.items():
        allrows = np.concatenate(lists) if n > 0 else np.zeros(0, dtype=np.int64)
        fetched[c] = iter(_row_values(table.columns[c], allrows) if n > 0 else [0] * len(allrows))
    for terms in plan:
        pred = []
        for c, op, rows, width in terms:
            vals = [next(fetched[c]) for _ in range(len(rows))]
            if table.dtypes[c] == F32:
                x = float(vals[0])
                pred.append(Term(c, RANGE, x, x + width))
            elif op == EQ:
                pred.append(Term(c, EQ, int(vals[0])))
            elif op == RANGE:
                x = int(vals[0])
                pred.append(Term(c, RANGE, x, x + max(1, int(width))))
            else:
                pred.append(Term(c, IN, values=tuple(int(v) for v in vals)))
        preds.append(pred)
    return preds


# ----------------------------------------------------------------- batched workload

def make_batched(ntables: int = 256, min_rows: int = 10_000, max_rows: int = 50_000_000,
                 nprobes: int = 4096, seed: int = 1004, device="cpu", key_domain: int = 1 << 15):
    """Many tables and a mixed request list for the batched form.

    Tables: rows log-uniform in [min_rows, max_rows]; 4-8 columns; column 0 an
    int32 join key Zipf(s) over `key_domain` values, the others int32 Zipf(s)
    over 2^20 values or float32 N(0,1), half and half; s uniform in [0.8, 1.5]
    per table.  Requests: 70 % predicate probes of 1-4 terms (50 % full scan,
    30 % a 1 % row sample, 20 % a 1 % sample of 4096-row blocks), 20 % HLL
    sketches (p = 12 or 14), 10 % joins between random table pairs on their
    key columns with a RANGE filter on each side.  Returns (tables, requests),
    each request a dict of plain data."""
    rng = np.random.default_rng(seed)
    g = _gen(seed, device)
    tables = []
    for t in range(ntables):
        n = int(math.exp(rng.uniform(math.log(min_rows), math.log(max_rows))))
        ncols = int(rng.integers(4, 9))
        s = float(rng.uniform(0.8, 1.5))
        cols = [zipf_column(n, s, key_domain, g, device)]
        dtypes, domains = [I32], [key_domain]
        for _ in range(ncols - 1):
            if rng.random() < 0.5:
                cols.append(zipf_column(n, s, 1 << 20, g, device))
                dtypes.append(I32)
                domains.append(1 << 20)
            else:
                cols.append(normal_column(n, g, device))
                dtypes.append(F32)
                domains.append(8.0)
        tables.append(Table(f"t{t}", cols, dtypes, domains))
    from .spec import BLOCKS, FULL, ROWS, Sample
    requests = []
    for i in range(nprobes):
        u = rng.random()
        t = int(rng.integers(0, ntables))
        if u < 0.7:
            preds = make_predicates(tables[t], 1, 1, 4, seed=seed * 1000 + i)
            v = rng.random()
            smp = Sample(FULL) if v < 0.5 else (Sample(ROWS, 0.01, 42) if v < 0.8 else Sample(BLOCKS, 0.01, 42, 4096))
            requests.append({"kind": "probe", "table": t, "preds": preds, "samples": [smp]})
        elif u < 0.9:
            requests.append({"kind": "ndv", "table": t, "col": int(rng.integers(0, len(tables[t].columns))),
                             "p": 12 if rng.random() < 0.5 else 14, "seed": 42})
        else:
            d = int(rng.integers(0, ntables))
            wf, wd = int(rng.integers(1, 1 << 20)), int(rng.integers(1, 1 << 20))
            fcol = [c for c in range(1, len(tables[t].columns)) if tables[t].dtypes[c] == I32]
            dcol = [c for c in range(1, len(tables[d].columns)) if tables[d].dtypes[c] == I32]
            fterms = [Term(fcol[0], RANGE, 0, wf)] if fcol else []
            dterms = [Term(dcol[0], RANGE, 0, wd)] if dcol else []
            requests.append({"kind": "join", "fact": t, "dim": d, "fact_terms": fterms, "dim_terms": dterms,
                             "key_domain": key_domain})
    _cdf_cache.clear()  # one table per (s, domain): do not keep them on the device
    return tables, requests
