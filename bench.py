#!/usr/bin/env python
"""Benchmark of the GACE probe path on GB300.

One step is the skew + correlation measurement: a 100M-row x 8-column table
(4 int32, 2 int64, 2 float32; Zipf s = 1.2 and a rho = 0.9 copula on two column
pairs, N(0,1) floats), 1024 conjunctive predicates of 1-4 terms counted on the
full table, 0.1 % / 1 % / 10 % row samples and a 1 % sample of 4096-row blocks
(seed 42) with per-term marginals and PCS, plus HyperLogLog (p = 14) of every
column.  value = rows measured per second, device-timed with CUDA events on the
stream the library launches on, inputs resident in HBM.

Also reported in the same line: the dominant kernel's roofline (live CUDA-event
times from the library's own tracing), the same metric end to end through the
C ABI from pinned host memory, single-probe scans against the HBM roofline, the
500M-row join probe, the CPU oracle timed on a bounded sample, the batched
form (4096 mixed requests over 256 tables in one batch) against one
synchronous call per request, and the served form under Poisson arrivals
(p50 / p99 latency and throughput) against the plain path at the same rates.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "probe rows/s & HBM % of peak; batched vs plain probes/s; p50/p99 probe ms"
WORKLOAD = ("skew_corr: 100M rows x 8 cols (4 i32, 2 i64, 2 f32), 1024 preds of 1-4 terms "
            "x {full, rows 0.1/1/10 %, blocks 4096 @ 1 %} with marginals + PCS, HLL p=14 x 8 cols")
SM_COUNT_FALLBACK = 152


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gace", "reference"], default="gace")
    ap.add_argument("--rows", type=int, default=100_000_000)
    ap.add_argument("--cpu-rows", type=int, default=250_000,
                    help="rows of the bounded sample the CPU oracle measures")
    ap.add_argument("--ref-rows", type=int, default=50_000,
                    help="rows per step of the reference arm (the oracle)")
    ap.add_argument("--no-extras", action="store_true", help="skip single-probe, join and e2e legs")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched and served legs")
    ap.add_argument("--serve-rates", default="1000,10000,50000,100000,200000",
                    help="Poisson arrival rates (requests/s) of the served leg")
    ap.add_argument("--serve-window", type=float, default=2.0, help="seconds of arrivals per rate")
    ap.add_argument("--serve-cap", type=int, default=20000, help="requests per rate at most")
    ap.add_argument("--case", default=None,
                    choices=["narrow_i32", "narrow_4xi32", "narrow_rows1pct", "wide_batch", "hll_i32",
                             "join_gather", "batch_mix", "batch_probes", "join_skew", "materialize"],
                    help="profiling driver: run one kernel family three times on a small (--rows) case")
    return ap.parse_args()


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return {"hbm_gbs": float(p["hbm_gbs"]), "sm_max_mhz": float(p.get("sm_max_mhz", 2070.0)),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "source": "fallback"}


# ----------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.idx)], stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = max(mx, float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- distributed

class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None

    def init(self, backend):
        if self.world > 1:
            import torch.distributed as dist

            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float, device) -> float:
        if not self.pg:
            return x
        import torch

        t = torch.tensor([x], dtype=torch.float64, device=device)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def done(self):
        if self.pg:
            self.pg.destroy_process_group()


# ----------------------------------------------------------------- workload

SAMPLES_SPEC = [("full", 0, 1.0, 0), ("rows", 1, 0.001, 0), ("rows", 1, 0.01, 0), ("rows", 1, 0.1, 0),
                ("blocks", 2, 0.01, 4096)]


def make_workload(n_rows, device, seed_offset=0):
    from workloads import Sample, make_predicates, make_skew_corr

    table = make_skew_corr(n=n_rows, seed=1002 + seed_offset, device=device)
    preds = make_predicates(table, 1024, 1, 4, seed=2002 + seed_offset)
    samples = [Sample(kind, rate, 42, block or 4096) for _, kind, rate, block in SAMPLES_SPEC]
    return table, preds, samples


def cpu_oracle_rate(table, preds, samples, rows: int):
    """Rows/s of the single-threaded oracle over the first `rows` rows of the
    same workload (every sample and every HLL sketch)."""
    import oracle

    oracle.build()
    host = [c[:rows].cpu().numpy() for c in table.columns]
    t0 = time.perf_counter()
    for s in samples:
        oracle.probe(host, table.dtypes, preds, s, marginals=True)
    for c in range(len(host)):
        oracle.hll_registers(host[c], table.dtypes[c], 14, 42)
    dt = time.perf_counter() - t0
    return rows / dt, dt


# ----------------------------------------------------------------- reference arm

def run_reference(args, d: Dist):
    if d.rank != 0:
        return
    import torch

    from workloads import make_predicates, make_skew_corr, Sample

    n = min(args.ref_rows, args.rows)
    table = make_skew_corr(n=n, seed=1002, device="cpu")
    preds = make_predicates(table, 1024, 1, 4, seed=2002)
    samples = [Sample(kind, rate, 42, block or 4096) for _, kind, rate, block in SAMPLES_SPEC]
    times = []
    for i in range(args.warmup + args.steps):
        _, dt = cpu_oracle_rate(table, preds, samples, n)
        if i >= args.warmup:
            times.append(dt)
    ms = 1000.0 * sum(times) / len(times)
    value = n / (ms / 1000.0)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "rows_per_step": n,
                   "note": "the reference is the single-threaded CPU oracle on a bounded sample"},
        "cpu_baseline": {"value": value, "unit": "rows/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {n} rows of the workload, every sample and sketch"},
        "e2e": {"value": value, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    del torch
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- GACE arm

def measured_traffic(fam, rows_per_launch):
    """DRAM bytes per launch of a kernel family from its committed ncu capture
    (profiles/roofline_traffic.json: bytes per row of the captured launches,
    scaled by rows), or None when there is none or the kernels' sources have
    changed since the capture."""
    import hashlib

    try:
        with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as f:
            rec = json.load(f)
        k = rec["kernels"][fam]
        h = hashlib.sha256()
        for src in rec["sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
    except (OSError, ValueError, KeyError):
        return None
    if h.hexdigest() != rec["sources_sha256"]:
        return None
    return k["bytes_per_row"] * rows_per_launch


def term_evals_per_row(preds):
    """Term evaluations one row of the batch costs, as the measurement plan
    counts them: 1 per EQ or RANGE term, k per IN list of k values."""
    from workloads import IN

    return sum(len(t.values) if t.op == IN else 1 for p in preds for t in p)


# The probe pipeline of one call: row-set masks, the rank pass of every
# rank-coded column (ranks and per-set rank histograms), the wide passes.
PROBE_PIPELINE = ("probe_setmask", "probe_rank", "probe_wide")


def roofline_of(stats, peaks, sms, steps, alu=None):
    """Roofline object of the step's dominant work.  When the wide probe pass
    is the family with the most device time, the probe pipeline as a whole
    (PROBE_PIPELINE): the batch's term evaluations (alu["evals"] per run)
    per second of the pipeline's device time, against the integer lane-op
    rate gace_calibrate_int measured on this GPU; traffic is the pipeline's
    DRAM bytes per step from the committed captures.  Otherwise the family's
    algorithmic bytes per second against the measured HBM copy rate."""
    fam, st = max(stats.items(), key=lambda kv: kv[1]["total_ms"])
    if fam == "probe_wide" and alu is not None:
        fams = [k for k in PROBE_PIPELINE if k in stats]
        sec = sum(stats[k]["total_ms"] for k in fams) / 1000.0
        traffic = 0.0
        for k in fams:
            t = measured_traffic(k, stats[k]["rows"] / max(1, stats[k]["launches"]))
            traffic = None if t is None or traffic is None else traffic + t * stats[k]["launches"] / steps
        achieved = alu["evals"] / sec / 1e12
        peak = alu["lane_ops_per_s"] / 1e12
        nominal = sms * 128 * peaks["sm_max_mhz"] * 1e6 / 1e12
        return "probe", {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                         "frac": achieved / peak, "traffic": traffic, "traffic_per": "step",
                         "algorithmic_bytes_per_step": sum(stats[k]["bytes"] for k in fams) / steps,
                         "work": "term evaluations (EQ 1, RANGE 1, IN-k k per row) of the whole batch",
                         "kernels": fams,
                         "device_ms_per_step": {k: stats[k]["total_ms"] / steps for k in fams},
                         "launches_per_step": {k: stats[k]["launches"] / steps for k in fams},
                         "peak_source": "measured: gace_calibrate_int kind 0 (32-bit xor/add lane ops) on this GPU",
                         "lane_ops_per_sm_clk": alu["lane_ops_per_s"] / (sms * peaks["sm_max_mhz"] * 1e6),
                         "range_tests_per_s_measured": alu["range_tests_per_s"],
                         "frac_of_range_test_rate": alu["evals"] / sec / alu["range_tests_per_s"],
                         "frac_of_nominal_128_lanes": achieved / nominal}
    sec = st["total_ms"] / 1000.0
    rows_per_launch = st["rows"] / max(1, st["launches"])
    traffic = measured_traffic(fam, rows_per_launch)
    algo_bytes = st["bytes"] / max(1, st["launches"])
    achieved = st["bytes"] / sec / 1e9
    return fam, {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                 "frac": achieved / peaks["hbm_gbs"], "traffic": traffic, "algorithmic_bytes_per_launch": algo_bytes,
                 "launches": st["launches"], "avg_launch_ms": st["total_ms"] / st["launches"]}


def run_gace(args, d: Dist):
    import numpy as np
    import torch

    import paper_2512_19750_gb300 as g

    dev = torch.device("cuda", d.local)
    torch.cuda.set_device(dev)  # before the process group, so that NCCL binds this rank's GPU
    d.init("nccl")
    peaks = load_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count or SM_COUNT_FALLBACK
    stream = torch.cuda.current_stream(dev)
    table, preds, samples = make_workload(args.rows, dev, seed_offset=d.rank)
    n = table.nrows
    table_bytes = int(sum(c.numel() * c.element_size() for c in table.columns))
    ctx = g.gace_create(d.local, stream=stream)
    tid = g.gace_load_columns(ctx, table.columns, borrow=True)
    batch = g.TermBatch(preds, table.dtypes)

    def step(table_id):
        res, marg = g.gace_probe_batch(ctx, table_id, preds, samples, table.dtypes, marginals=True,
                                       batch=batch)
        regs = [g.gace_ndv(ctx, table_id, c, 14, 42) for c in range(len(table.columns))]
        return res, marg, regs

    for _ in range(args.warmup):
        step(tid)
    g.gace_stats_reset(ctx, time_kernels=True)
    clk = ClockSampler(d.local)
    d.barrier()
    torch.cuda.synchronize(dev)
    clk.start()
    t_a = torch.cuda.Event(enable_timing=True)
    t_b = torch.cuda.Event(enable_timing=True)
    t_a.record(stream)
    for _ in range(args.steps):
        step(tid)
    t_b.record(stream)
    torch.cuda.synchronize(dev)
    d.barrier()
    clocks = clk.stop()
    ms_total = d.max(t_a.elapsed_time(t_b), dev)
    allstats = g.gace_stats_read(ctx)
    # kernel families only; the host phases of the calls are reported apart
    stats = {k: v for k, v in allstats.items() if not k.startswith("host_")}
    host_phases = {k[len("host_"):]: round(v["total_ms"] / args.steps, 3)
                   for k, v in allstats.items() if k.startswith("host_")}
    ms_per_step = ms_total / args.steps
    value = d.world * n * args.steps / (ms_total / 1000.0)
    gpu_launches = sum(s["launches"] for s in stats.values())
    alu = {"evals": float(n) * term_evals_per_row(preds) * args.steps,
           "lane_ops_per_s": g.gace_calibrate_int(ctx, 0, 50),
           "range_tests_per_s": g.gace_calibrate_int(ctx, 1, 50)}
    fam, roof = roofline_of(stats, peaks, sms, args.steps, alu)
    roof["kernel"] = fam
    roof["peak_source"] = roof.get("peak_source", f"MEASURED_PEAKS.json hbm_gbs ({peaks['source']})")
    kernels = {k: {"launches": v["launches"], "total_ms": round(v["total_ms"], 3),
                   "share": round(v["total_ms"] / max(1e-9, sum(x["total_ms"] for x in stats.values())), 4)}
               for k, v in stats.items()}

    cpu = None
    if d.rank == 0 and d.world == 1:
        m = min(args.cpu_rows, n)
        rate, dt = cpu_oracle_rate(table, preds, samples, m)
        cpu = {"value": rate, "unit": "rows/s", "cores": 1, "kind": "oracle",
               "sample": f"first {m} rows of the same table and batch (all 5 row sets, marginals, "
                         f"8 HLL sketches), single-threaded, {dt:.1f} s"}

    extras = {}
    if not args.no_extras:
        extras["single_probe"] = single_probes(g, ctx, tid, table, peaks, stream)
        extras["plain_small"] = plain_small_leg(g, ctx, dev, peaks, stream)
        extras["stability"] = stability_leg(g, ctx, tid, table)
        extras["e2e"], extras["overhead"] = e2e_leg(g, ctx, table, preds, samples, batch, args, stream)
    g.gace_unload(ctx, tid)
    if not args.no_extras:
        del table
        torch.cuda.empty_cache()
        extras["join"] = join_leg(g, ctx, dev, peaks, stream)
    if not args.no_batch and d.world == 1:
        extras["batched"] = batched_leg(g, ctx, dev, args)
        extras["served"] = served_leg(g, ctx, dev, args)
    g.gace_destroy(ctx)

    d.barrier()
    if d.rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": d.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "rows": n, "predicates": len(preds),
                       "terms": sum(len(p) for p in preds), "row_sets": len(samples),
                       "table_bytes": table_bytes,
                       "l2": "inputs (4 GB) larger than the 129 MB L2; no flush needed",
                       "parallelism": f"replicas x{d.world}"},
            "roofline": roof,
            "kernels": kernels,
            "host_ms_per_step": host_phases,
            "cpu_baseline": cpu,
            "e2e": extras.get("e2e"),
            "gpu_launches": gpu_launches,
            "clocks": clocks,
            "single_probe": extras.get("single_probe"),
            "plain_small": extras.get("plain_small"),
            "join": extras.get("join"),
            "stability": extras.get("stability"),
            "overhead": extras.get("overhead"),
            "batched": extras.get("batched"),
            "served": extras.get("served"),
        }
        print(json.dumps(line), flush=True)
    d.done()


def kernel_stats(g, ctx):
    """The context's statistics of kernel families (without the host phases
    of the calls, which timing also records)."""
    return {k: v for k, v in g.gace_stats_read(ctx).items() if not k.startswith("host_")}


def _timed_calls(g, ctx, fn, reps):
    g.gace_stats_reset(ctx, time_kernels=True)
    for _ in range(reps):
        fn()
    return kernel_stats(g, ctx)


def sampled_estimates(g, ctx, tid, dtypes, preds, rate, seeds, block_rows=0):
    """sel of every predicate and PCS of every 2-term predicate for each seed
    of a row (or block) sample at one rate: arrays [seeds][preds].  Eight
    samples per call (the probe's row sets)."""
    from workloads import BLOCKS, ROWS, Sample

    sel, pcs = [], []
    for b in range(0, len(seeds), 8):
        smp = [Sample(BLOCKS, rate, s, block_rows) if block_rows else Sample(ROWS, rate, s) for s in seeds[b:b + 8]]
        res, _ = g.gace_probe_batch(ctx, tid, preds, smp, dtypes)
        sel.extend(res["sel"][:len(smp)].tolist())
        pcs.extend(res["pcs"][:len(smp)].tolist())
    return np.array(sel), np.array(pcs)


def cv(x):
    """Coefficient of variation across seeds (axis 0), NaN where the mean is 0."""
    m = x.mean(axis=0)
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(m != 0, x.std(axis=0) / m, np.nan)


def stability_leg(g, ctx, tid, table):
    """Estimation stability vs budget (the paper's Experiment B): the
    coefficient of variation over 100 seeds of sel(A and B) and of PCS for
    two-column conjunctions (a correlated pair, c0/c1, and an independent
    one, c2/c6), per row-sample rate and for 4096-row block samples."""
    from workloads import RANGE, Term

    preds = [[Term(0, RANGE, 0, 40), Term(1, RANGE, 0, 40)], [Term(2, RANGE, 0, 40), Term(6, RANGE, -0.5, 0.5)]]
    seeds = list(range(1, 101))
    out = {}
    for label, rate, block in (("rows 0.1%", 0.001, 0), ("rows 1%", 0.01, 0), ("rows 10%", 0.1, 0),
                               ("blocks 1%", 0.01, 4096), ("blocks 10%", 0.1, 4096)):
        t0 = time.perf_counter()
        sel, pcs = sampled_estimates(g, ctx, tid, table.dtypes, preds, rate, seeds, block)
        out[label] = {"cv_sel": [round(float(x), 5) for x in cv(sel)], "cv_pcs": [round(float(x), 5) for x in cv(pcs)],
                      "mean_pcs": [round(float(x), 4) for x in np.nanmean(pcs, axis=0)],
                      "wall_ms_100_seeds": round(1000 * (time.perf_counter() - t0), 2)}
    out["predicates"] = "A and B: c0 in [0,40) and c1 in [0,40) (copula rho 0.9); c2 in [0,40) and c6 in [-0.5,0.5)"
    return out


def single_probes(g, ctx, tid, table, peaks, stream):
    """One-predicate full scans (the gate's single probes): HBM roofline."""
    from workloads import FULL, F32, RANGE, Sample, Term

    out = {}
    n = table.nrows
    cases = {"1 x int32 RANGE": [0], "1 x int64 RANGE": [4], "2 x int32 RANGE (PCS)": [0, 1],
             "4 x int32 RANGE": [0, 1, 2, 3]}
    for name, cols in cases.items():
        pred = [[Term(c, RANGE, 0, 1000) if table.dtypes[c] != F32 else Term(c, RANGE, -1.0, 1.0)
                 for c in cols]]
        b = g.TermBatch(pred, table.dtypes)
        g.gace_probe_batch(ctx, tid, pred, [Sample(FULL)], table.dtypes, batch=b)
        st = _timed_calls(g, ctx, lambda: g.gace_probe_batch(ctx, tid, pred, [Sample(FULL)], table.dtypes,
                                                             batch=b), 10)
        k = st["probe_narrow"]
        ms = k["total_ms"] / k["launches"]
        gbs = k["bytes"] / k["launches"] / (ms / 1000.0) / 1e9
        out[name] = {"kernel_ms": round(ms, 4), "rows_per_s": n / (ms / 1000.0), "gbs": gbs,
                     "frac_of_measured_hbm": gbs / peaks["hbm_gbs"]}
    return out


def plain_small_leg(g, ctx, dev, peaks, stream):
    """The plain small probe: 1M rows x 4 int32 (16 MB), 64 predicates of 1-3
    terms on the full table and a 1 % row sample (seed 42) with marginals and
    PCS, plus HyperLogLog (p = 12) of the four columns.  The table fits in the
    129 MB L2, so a step is latency-bound: microseconds per step (median of
    50 after 5 warm-up, CUDA events on the library's stream around the
    synchronous calls), and the same with a 256 MB write before each step
    (outside the timed interval) that evicts the table from L2, for HBM bytes
    per second."""
    import torch

    from workloads import FULL, ROWS, Sample, make_plain_small, make_predicates

    t = make_plain_small(seed=1001, device=dev)
    preds = make_predicates(t, 64, 1, 3, seed=2001)
    samples = [Sample(FULL), Sample(ROWS, 0.01, 42)]
    tid = g.gace_load_columns(ctx, t.columns, borrow=True)
    batch = g.TermBatch(preds, t.dtypes)

    def step():
        g.gace_probe_batch(ctx, tid, preds, samples, t.dtypes, marginals=True, batch=batch)
        for c in range(4):
            g.gace_ndv(ctx, tid, c, 12, 42)

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    algo_bytes = 2 * t.nrows * 4 * 4  # the probe reads 4 columns, the 4 sketches read them again
    out = {"workload": "1M rows x 4 int32 (c0 U[0,1e6), c1 Zipf(1.1,1e4), c2 = 7 c1 + U[0,50), c3 U[0,100)); "
                       "64 preds of 1-3 terms x {full, rows 1 % seed 42} with marginals + PCS; HLL p=12 x 4"}
    for mode in ("l2_resident", "l2_flushed"):
        times = []
        g.gace_stats_reset(ctx, time_kernels=True)
        for i in range(55):
            if mode == "l2_flushed":
                flush.fill_(i & 0xFF)
            if i == 5:
                g.gace_stats_reset(ctx, time_kernels=True)
            torch.cuda.synchronize(dev)
            a.record(stream)
            step()
            b.record(stream)
            torch.cuda.synchronize(dev)
            if i >= 5:
                times.append(a.elapsed_time(b))
        st = kernel_stats(g, ctx)
        kern_us = 1000.0 * sum(v["total_ms"] for v in st.values()) / 50
        us = 1000.0 * statistics.median(times)
        entry = {"us_per_step": us, "us_per_probe_call": None, "kernel_us_per_step": kern_us,
                 "kernels": {k: round(1000.0 * v["total_ms"] / 50, 2) for k, v in st.items()}}
        if mode == "l2_flushed":
            entry["kernel_gbs"] = algo_bytes / (kern_us * 1e-6) / 1e9
            entry["kernel_frac_of_measured_hbm"] = entry["kernel_gbs"] / peaks["hbm_gbs"]
        out[mode] = entry
    # one synchronous probe call alone (no sketches), L2-resident
    times = []
    for i in range(55):
        torch.cuda.synchronize(dev)
        a.record(stream)
        g.gace_probe_batch(ctx, tid, preds, samples, t.dtypes, marginals=True, batch=batch)
        b.record(stream)
        torch.cuda.synchronize(dev)
        if i >= 5:
            times.append(a.elapsed_time(b))
    out["l2_resident"]["us_per_probe_call"] = 1000.0 * statistics.median(times)
    g.gace_unload(ctx, tid)
    del flush, t
    torch.cuda.empty_cache()
    return out


def e2e_leg(g, ctx, table, preds, samples, batch, args, stream):
    """The same step through the C ABI from pinned host memory: the table
    registered with its copy deferred to the probe (which streams it in row
    chunks while its passes run on the chunks already copied), the probe
    batch and the 8 sketches, results read back."""
    import torch

    host = [c.cpu().pin_memory() for c in table.columns]
    h2d = sum(h.numel() * h.element_size() for h in host)

    def once():
        t = g.gace_load_columns(ctx, host, copy_on_first_probe=True)
        res, marg = g.gace_probe_batch(ctx, t, preds, samples, table.dtypes, marginals=True, batch=batch)
        regs = [g.gace_ndv(ctx, t, c, 14, 42) for c in range(len(table.columns))]
        g.gace_unload(ctx, t)
        return res, marg, regs

    for _ in range(max(3, args.warmup)):  # warm-up steps, as for the device-timed step
        res, marg, regs = once()
    d2h = res.nbytes + marg.nbytes + sum(r[0].nbytes for r in regs)
    reps = max(3, min(args.steps, 7))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    marks = []
    for _ in range(reps):
        once()
        marks.append(time.perf_counter())
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / reps
    per_step = [1e3 * (b - a) for a, b in zip([t0] + marks[:-1], marks)]
    # where one more step's time goes (outside the timed steps)
    ph = []
    for _ in range(2):
        torch.cuda.synchronize()
        ta = time.perf_counter()
        t = g.gace_load_columns(ctx, host, copy_on_first_probe=True)
        tb = time.perf_counter()
        g.gace_probe_batch(ctx, t, preds, samples, table.dtypes, marginals=True, batch=batch)
        tc = time.perf_counter()
        for c in range(len(table.columns)):
            g.gace_ndv(ctx, t, c, 14, 42)
        td = time.perf_counter()
        g.gace_unload(ctx, t)
        torch.cuda.synchronize()
        te = time.perf_counter()
        ph.append({"load": 1e3 * (tb - ta), "probe_with_h2d": 1e3 * (tc - tb), "sketches": 1e3 * (td - tc),
                   "unload": 1e3 * (te - td)})
    # The value is from the median step: the host-to-device copies share the
    # machine's host links with other jobs, and one step in a few has been
    # seen to stall for 100-200 ms; the mean is reported beside it.
    med = statistics.median(per_step) / 1000.0
    out = {"value": table.nrows / med, "unit": "rows/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "ms_per_step": med * 1000.0, "mean_ms_per_step": dt * 1000.0,
           "statistic": "median step", "steps": reps,
           "per_step_ms": [round(x, 2) for x in per_step],
           "phases_ms": {k: round(min(p[k] for p in ph), 3) for k in ph[0]}}
    overhead = overhead_leg(g, ctx, host, table.dtypes)
    del host
    return out, overhead


def overhead_leg(g, ctx, host, dtypes):
    """Probe overhead decomposition (the paper's Experiment A) for tables that
    are not resident: H2D of the columns from pinned host memory (key-only:
    the two referenced columns; full-row: all eight), the kernel, and the
    read-back with the host's reduction into results, for N = 1e4 .. 1e8 rows
    of one two-term probe (median of 3)."""
    from workloads import FULL, RANGE, Sample, Term

    preds = [[Term(0, RANGE, 0, 40), Term(1, RANGE, 0, 40)]]
    out = {}
    for mode, cols in (("key-only", [0, 1]), ("full-row", list(range(len(host))))):
        out[mode] = {}
        for n in (10**4, 10**5, 10**6, 10**7, 10**8):
            if n > host[0].numel():
                continue
            ph = []
            for _ in range(3):
                t0 = time.perf_counter()
                tid = g.gace_load_columns(ctx, [host[c][:n] for c in cols])
                t1 = time.perf_counter()
                g.gace_stats_reset(ctx, time_kernels=True)
                g.gace_probe_batch(ctx, tid, preds, [Sample(FULL)], [dtypes[c] for c in cols])
                t2 = time.perf_counter()
                kern = sum(v["total_ms"] for v in kernel_stats(g, ctx).values())
                g.gace_unload(ctx, tid)
                ph.append(((t1 - t0) * 1e3, kern, (t2 - t1) * 1e3 - kern))
            h2d, kern, rest = (statistics.median(x[i] for x in ph) for i in range(3))
            out[mode][f"{n:.0e}"] = {"h2d_ms": round(h2d, 4), "kernel_ms": round(kern, 4),
                                     "d2h_and_reduction_ms": round(rest, 4), "total_ms": round(h2d + kern + rest, 4),
                                     "transfer_share": round(h2d / (h2d + kern + rest), 3)}
    return out


def join_leg(g, ctx, dev, peaks, stream):
    """Join probe: 500M-row fact (Zipf FK over 10M keys) x 10M-row dimension,
    filters at 1 % and 10 %, gather method; plus the 3-table chain."""
    import torch

    from workloads import RANGE, Term, make_join

    f, dm, d2 = make_join(seed=1003, device=dev)
    fid = g.gace_load_columns(ctx, f.columns, borrow=True)
    did = g.gace_load_columns(ctx, dm.columns, borrow=True)
    d2id = g.gace_load_columns(ctx, d2.columns, borrow=True)
    out = {}
    for w in (10, 100):
        F = g.JoinSideSpec(fid, 0, [Term(1, RANGE, 0, w)], f.dtypes)
        D = g.JoinSideSpec(did, 0, [Term(1, RANGE, 0, w)], dm.dtypes)
        g.gace_join_card(ctx, F, D, 10_000_000)
        st = _timed_calls(g, ctx, lambda: g.gace_join_card(ctx, F, D, 10_000_000), 5)
        tot = sum(v["total_ms"] for v in st.values()) / 5
        gk = st["join_gather"]
        gms = gk["total_ms"] / gk["launches"]
        gbs = gk["bytes"] / gk["launches"] / (gms / 1000.0) / 1e9
        out[f"2-table sel {w / 10:.0f}%"] = {
            "kernels_ms": round(tot, 4), "fact_rows_per_s": f.nrows / (tot / 1000.0),
            "gather_gbs": gbs, "gather_frac_of_measured_hbm": gbs / peaks["hbm_gbs"]}
    F = g.JoinSideSpec(fid, 0, [Term(1, RANGE, 0, 100)], f.dtypes)
    D = g.JoinSideSpec(did, 0, [Term(1, RANGE, 0, 500)], dm.dtypes)
    D2 = g.JoinSideSpec(d2id, 0, [Term(1, RANGE, 0, 500)], d2.dtypes)
    st = _timed_calls(g, ctx, lambda: g.gace_join_card(ctx, F, D, 10_000_000, D2, 1_000_000, 3), 3)
    out["3-table chain"] = {"kernels_ms": round(sum(v["total_ms"] for v in st.values()) / 3, 4)}
    for t in (fid, did, d2id):
        g.gace_unload(ctx, t)
    del f, dm, d2
    torch.cuda.empty_cache()
    return out


def to_gace_requests(g, tids, tables, reqs):
    """Request objects of the library from the generated mixed workload."""
    out = []
    for r in reqs:
        if r["kind"] == "probe":
            t = tables[r["table"]]
            out.append(g.ProbeRequest(tids[r["table"]], r["preds"], r["samples"], t.dtypes, marginals=True))
        elif r["kind"] == "ndv":
            out.append(g.NdvRequest(tids[r["table"]], r["col"], r["p"], r["seed"]))
        else:
            f, d = tables[r["fact"]], tables[r["dim"]]
            out.append(g.JoinRequest(g.JoinSideSpec(tids[r["fact"]], 0, r["fact_terms"], f.dtypes),
                                     g.JoinSideSpec(tids[r["dim"]], 0, r["dim_terms"], d.dtypes),
                                     r["key_domain"]))
    return out


def request_bytes(tables, reqs):
    """Algorithmic bytes of each request run alone: the referenced columns of
    every table it scans, once."""
    out = []
    for r in reqs:
        if r["kind"] == "probe":
            t = tables[r["table"]]
            cols = {term.col for p in r["preds"] for term in p}
            out.append(t.nrows * sum(t.columns[c].element_size() for c in cols))
        elif r["kind"] == "ndv":
            t = tables[r["table"]]
            out.append(t.nrows * t.columns[r["col"]].element_size())
        else:
            b = 0
            for side, terms in ((r["fact"], r["fact_terms"]), (r["dim"], r["dim_terms"])):
                t = tables[side]
                cols = {0} | {term.col for term in terms}
                b += t.nrows * sum(t.columns[c].element_size() for c in cols)
            out.append(b)
    return out


def shared_scan_bytes(tables, reqs):
    """Algorithmic bytes of the batch when every table is scanned once for all
    the requests on it: per table, its rows times the widths of the union of
    the columns its requests reference."""
    cols = {}
    for r in reqs:
        if r["kind"] == "probe":
            cols.setdefault(r["table"], set()).update(term.col for p in r["preds"] for term in p)
        elif r["kind"] == "ndv":
            cols.setdefault(r["table"], set()).add(r["col"])
        else:
            for side, terms in ((r["fact"], r["fact_terms"]), (r["dim"], r["dim_terms"])):
                cols.setdefault(side, set()).update({0} | {term.col for term in terms})
    return sum(tables[t].nrows * sum(tables[t].columns[c].element_size() for c in cs) for t, cs in cols.items())


def batched_leg(g, ctx, dev, args):
    """4096 mixed requests over 256 tables: one batch (persistent kernel,
    graph, autotuned chunk and grid) against one synchronous call per request
    and against the served form with every request arriving at once."""
    import numpy as np
    import torch

    from workloads import make_batched

    tables, reqs = make_batched(ntables=256, min_rows=10_000, max_rows=50_000_000, nprobes=4096, seed=1004,
                                device=dev)
    tids = [g.gace_load_columns(ctx, t.columns, borrow=True) for t in tables]
    nbytes = sum(request_bytes(tables, reqs))
    shared = shared_scan_bytes(tables, reqs)
    n = len(reqs)
    g.gace_stats_reset(ctx)
    g.gace_tune_batch(ctx, to_gace_requests(g, tids, tables, reqs))
    tuned = g.gace_stats_read(ctx)
    fuse_ms = {k: round(v["total_ms"], 3) for k, v in tuned.items() if k.startswith("tune_batch_")}
    breqs = g.RequestArray(to_gace_requests(g, tids, tables, reqs))  # marshalled once, run five times
    for _ in range(2):
        g.gace_run_batch(ctx, breqs)
    g.gace_stats_reset(ctx, time_kernels=True)
    walls = []
    for _ in range(5):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        g.gace_run_batch(ctx, breqs)
        walls.append(time.perf_counter() - t0)
    st = g.gace_stats_read(ctx)
    batch_ms = st["batch"]["total_ms"] / max(1, st["batch"]["launches"])
    host_ms = {k[len("host_batch_"):]: round(v["total_ms"] / max(1, v["launches"]), 3)
               for k, v in st.items() if k.startswith("host_batch_")}
    wall = float(np.median(walls))
    zero = np.zeros(n, dtype=np.uint64)
    plain_done, plain_st = g.gace_serve_replay(ctx, to_gace_requests(g, tids, tables, reqs), zero, mode=1)
    plain_wall = float(plain_done.max()) / 1e9
    # the plain path's device time alone: one launch sequence per request with
    # the host's waits between requests removed (what an asynchronous plain
    # path could reach at best)
    g.gace_stats_reset(ctx, time_kernels=True)
    g.gace_serve_replay(ctx, to_gace_requests(g, tids, tables, reqs), zero, mode=1)
    plain_dev_s = sum(v["total_ms"] for v in kernel_stats(g, ctx).values()) / 1000.0
    g.gace_stats_reset(ctx)
    # plain-async: the same synchronous calls spread over four contexts (one
    # host thread and stream each), so that calls overlap on the GPU
    nasync = 4
    actxs = [g.gace_create(dev.index or 0) for _ in range(nasync)]
    try:
        atids = [[g.gace_load_columns(c, t.columns, borrow=True) for t in tables] for c in actxs]
        areqs = g.RequestArray([to_gace_requests(g, atids[i % nasync], tables, [r])[0] for i, r in enumerate(reqs)])
        g.gace_run_plain_async(actxs, areqs)  # warm-up
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        async_st = g.gace_run_plain_async(actxs, areqs)
        async_wall = time.perf_counter() - t0
    finally:
        for c in actxs:
            g.gace_destroy(c)
    # no result caches: the warm-up run would answer the timed run's requests
    g.gace_serve_start(ctx, sketch_cache=-1, probe_cache=-1)
    g.gace_serve_replay(ctx, to_gace_requests(g, tids, tables, reqs), zero, mode=0)  # warm-up
    served_done, served_st = g.gace_serve_replay(ctx, to_gace_requests(g, tids, tables, reqs), zero, mode=0)
    g.gace_serve_stop(ctx)
    served_wall = float(served_done.max()) / 1e9
    # the same batch with the context's resident store (120 GB): 1 % row and
    # 1 % block samples of every table materialised first, sketches kept by a
    # first run; the plain path reads the same store
    from workloads import BLOCKS, ROWS, Sample
    g.gace_resident_configure(ctx, 120 << 30)
    for tid in tids:
        for smp in (Sample(ROWS, 0.01, 42), Sample(BLOCKS, 0.01, 42, 4096)):
            g.gace_resident_prefetch(ctx, tid, smp)
    rreqs = g.RequestArray(to_gace_requests(g, tids, tables, reqs))
    for _ in range(2):
        g.gace_run_batch(ctx, rreqs)
    rwalls = []
    for _ in range(5):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        g.gace_run_batch(ctx, rreqs)
        rwalls.append(time.perf_counter() - t0)
    rwall = float(np.median(rwalls))
    rplain_done, rplain_st = g.gace_serve_replay(ctx, to_gace_requests(g, tids, tables, reqs), zero, mode=1)
    rplain_wall = float(rplain_done.max()) / 1e9
    rstore = g.gace_resident_stats_read(ctx)
    g.gace_resident_configure(ctx, 0)
    for t in tids:
        g.gace_unload(ctx, t)
    rows = sum(t.nrows for t in tables)
    del tables
    torch.cuda.empty_cache()
    return {
        "workload": "256 tables, rows log-uniform [1e4, 5e7]; 4096 requests (70% predicate probes, 20% HLL, "
                    "10% joins)",
        "requests": n, "table_rows": rows, "request_bytes": nbytes,
        "batched_probes_per_s": n / wall, "batched_ms": wall * 1000.0, "batch_graph_ms": batch_ms,
        "batch_host_phases_ms": host_ms,
        "tuned_ms_by_fusion_rule": fuse_ms,
        "plain_probes_per_s": n / plain_wall, "plain_ms": plain_wall * 1000.0,
        "plain_device_only_probes_per_s": n / plain_dev_s, "plain_device_only_ms": plain_dev_s * 1000.0,
        "plain_async_probes_per_s": n / async_wall, "plain_async_ms": async_wall * 1000.0,
        "plain_async": f"the synchronous calls on {nasync} contexts, one host thread and stream each",
        "served_at_once_probes_per_s": n / served_wall, "served_at_once_ms": served_wall * 1000.0,
        "batched_vs_plain": plain_wall / wall,
        "batched_gbs": nbytes / wall / 1e9,
        "shared_scan_bytes": shared,
        "batched_gbs_shared_scan": shared / wall / 1e9,
        "resident_store": {"batched_probes_per_s": n / rwall, "batched_ms": rwall * 1000.0,
                           "plain_probes_per_s": n / rplain_wall, "plain_ms": rplain_wall * 1000.0,
                           "batched_vs_plain": rplain_wall / rwall, "store": rstore,
                           "ok": bool((rplain_st == 0).all())},
        "all_ok": bool((plain_st == 0).all() and (served_st == 0).all() and async_st == [0] * n),
        "plain": "one synchronous call per request (probe / ndv / join_card) from a native loop",
    }


def served_leg(g, ctx, dev, args):
    """Open-loop Poisson arrivals of the config-4 mix over 64 tables of 1M to
    200M rows, served (continuous batching) and plain (one synchronous call
    per request in arrival order) at each rate: p50 / p99 latency and
    throughput, in three configurations:
      no_caches       neither side keeps anything between requests (the served
                      form's sketch and count caches off, no resident store):
                      continuous batching alone;
      resident_120gb  both sides with the context's resident store (120 GB):
                      1 % and 10 % row samples and 1 % block samples of every
                      table materialised before the run, sketches kept as they
                      are computed (the served form's host caches off);
      resident_256mb  a 256 MB store (a third of the 1 % samples the mix reads),
                      served at one rate, samples admitted on first use:
                      admission and eviction under pressure."""
    import numpy as np
    import torch

    from workloads import BLOCKS, ROWS, Sample, make_batched

    rates = [int(r) for r in args.serve_rates.split(",") if r]
    nmax = int(max(rates) * args.serve_window)
    tables, reqs = make_batched(ntables=64, min_rows=1_000_000, max_rows=200_000_000,
                                nprobes=min(nmax, args.serve_cap), seed=1005, device=dev)
    tids = [g.gace_load_columns(ctx, t.columns, borrow=True) for t in tables]
    rb = np.array(request_bytes(tables, reqs), dtype=np.float64)
    out = {"workload": "64 tables, rows log-uniform [1e6, 2e8], the config-4 request mix",
           "table_rows": sum(t.nrows for t in tables), "mean_request_bytes": float(rb.mean()),
           "window_s": args.serve_window, "cap_requests": args.serve_cap}

    def stats(arrival, done, st):
        lat = (done.astype(np.float64) - arrival.astype(np.float64)) / 1e6
        srt = np.sort(lat)
        k = len(srt)
        p50 = float(srt[max(0, math.ceil(0.50 * k) - 1)])
        p99 = float(srt[max(0, math.ceil(0.99 * k) - 1)])
        return {"p50_ms": p50, "p99_ms": p99, "throughput_per_s": k / (float(done.max()) / 1e9),
                "ok": bool((st == 0).all())}

    def sweep(rate_list, with_plain, label):
        res = {}
        rng = np.random.default_rng(7)
        for rate in rate_list:
            n = min(int(rate * args.serve_window), args.serve_cap, len(reqs))
            gaps = rng.exponential(1e9 / rate, n)
            arrival = np.cumsum(gaps).astype(np.uint64)
            sub = reqs[:n]
            entry = {"requests": n}
            g.gace_serve_start(ctx, sketch_cache=-1, probe_cache=-1)
            done, st = g.gace_serve_replay(ctx, to_gace_requests(g, tids, tables, sub), arrival, mode=0)
            g.gace_serve_stop(ctx)
            entry["served"] = stats(arrival, done, st)
            if with_plain:
                done, st = g.gace_serve_replay(ctx, to_gace_requests(g, tids, tables, sub), arrival, mode=1)
                entry["plain"] = stats(arrival, done, st)
            res[str(rate)] = entry
        return res

    # warm-up of both paths
    warm = to_gace_requests(g, tids, tables, reqs[:64])
    g.gace_serve_replay(ctx, warm, np.zeros(len(warm), dtype=np.uint64), mode=1)
    out["no_caches"] = sweep(rates, True, "no_caches")

    g.gace_resident_configure(ctx, 120 << 30)
    t0 = time.perf_counter()
    for tid in tids:
        for smp in (Sample(ROWS, 0.01, 42), Sample(ROWS, 0.1, 42), Sample(BLOCKS, 0.01, 42, 4096)):
            g.gace_resident_prefetch(ctx, tid, smp)
    prefetch_s = time.perf_counter() - t0
    g.gace_serve_replay(ctx, to_gace_requests(g, tids, tables, reqs), np.zeros(len(reqs), dtype=np.uint64),
                        mode=1)  # computes (and keeps) the sketches the mix asks for
    out["resident_120gb"] = sweep(rates, True, "resident_120gb")
    out["resident_120gb"]["store"] = dict(g.gace_resident_stats_read(ctx), prefetch_s=round(prefetch_s, 3))

    g.gace_resident_configure(ctx, 256 << 20)
    out["resident_256mb"] = sweep([rates[min(1, len(rates) - 1)]], False, "resident_256mb")
    out["resident_256mb"]["store"] = g.gace_resident_stats_read(ctx)
    # the same budget admitting a sample only at its fourth use: less churn
    g.gace_resident_configure(ctx, 256 << 20, admit_after=4)
    out["resident_256mb_admit4"] = sweep([rates[min(1, len(rates) - 1)]], False, "resident_256mb_admit4")
    out["resident_256mb_admit4"]["store"] = g.gace_resident_stats_read(ctx)
    g.gace_resident_configure(ctx, 0)
    for t in tids:
        g.gace_unload(ctx, t)
    del tables
    torch.cuda.empty_cache()
    return out


def run_case(args):
    """Small single-kernel cases for profiler captures (inputs above the L2
    size, a few GB on the device at most)."""
    import torch

    import paper_2512_19750_gb300 as g
    from workloads import FULL, RANGE, ROWS, Sample, Term, make_join, make_predicates

    dev = torch.device("cuda:0")
    ctx = g.gace_create(0, stream=torch.cuda.current_stream())
    if args.case == "join_gather":
        f, dm, _ = make_join(n_fact=args.rows, n_dim=10_000_000, n_dim2=1000, seed=1003, device=dev)
        fid = g.gace_load_columns(ctx, f.columns, borrow=True)
        did = g.gace_load_columns(ctx, dm.columns, borrow=True)
        F = g.JoinSideSpec(fid, 0, [Term(1, RANGE, 0, 100)], f.dtypes)
        D = g.JoinSideSpec(did, 0, [Term(1, RANGE, 0, 100)], dm.dtypes)
        for _ in range(3):
            out = g.gace_join_card(ctx, F, D, 10_000_000)
        print(json.dumps({"case": args.case, "rows": args.rows, "card": out["card"]}))
        g.gace_destroy(ctx)
        return
    if args.case == "batch_probes":
        # the config-4 probe requests over 16 tables of 1e6..5e7 rows (about 3 GB)
        from workloads import make_batched
        tables, reqs = make_batched(ntables=16, min_rows=1_000_000, max_rows=50_000_000, nprobes=600, seed=1005,
                                    device=dev)
        reqs = [r for r in reqs if r["kind"] == "probe"]
        tids = [g.gace_load_columns(ctx, t.columns, borrow=True) for t in tables]
        for _ in range(2):
            st = g.gace_run_batch(ctx, to_gace_requests(g, tids, tables, reqs))
        for r in reqs[:20]:  # the same probes one by one, for the plain kernels
            g.gace_probe_batch(ctx, tids[r["table"]], r["preds"], r["samples"], tables[r["table"]].dtypes)
        print(json.dumps({"case": args.case, "requests": len(reqs), "ok": st == [0] * len(reqs)}))
        g.gace_destroy(ctx)
        return
    if args.case == "join_skew":
        # fact and dimension of 40M rows each, keys Zipf(1.2) over 2^15 values
        from workloads import I32, Table, uniform_int_column, zipf_column
        from workloads.gen import _gen
        gen = _gen(1006, dev)
        n = args.rows
        f = Table("f", [zipf_column(n, 1.2, 1 << 15, gen, dev), uniform_int_column(n, 0, 1000, gen, dev)], [I32, I32])
        d = Table("d", [zipf_column(n, 1.2, 1 << 15, gen, dev), uniform_int_column(n, 0, 1000, gen, dev)], [I32, I32])
        fid = g.gace_load_columns(ctx, f.columns, borrow=True)
        did = g.gace_load_columns(ctx, d.columns, borrow=True)
        F = g.JoinSideSpec(fid, 0, [Term(1, RANGE, 0, 500)], f.dtypes)
        D = g.JoinSideSpec(did, 0, [Term(1, RANGE, 0, 500)], d.dtypes)
        for _ in range(3):
            out = g.gace_join_card(ctx, F, D, 1 << 15)
        print(json.dumps({"case": args.case, "rows": n, "card": out["card"]}))
        g.gace_destroy(ctx)
        return
    if args.case == "batch_mix":
        # the config-4 request mix over 32 tables of 1e5..2e7 rows (about 2 GB)
        from workloads import make_batched
        tables, reqs = make_batched(ntables=32, min_rows=100_000, max_rows=20_000_000, nprobes=512, seed=1004,
                                    device=dev)
        tids = [g.gace_load_columns(ctx, t.columns, borrow=True) for t in tables]
        for _ in range(2):
            st = g.gace_run_batch(ctx, to_gace_requests(g, tids, tables, reqs))
        print(json.dumps({"case": args.case, "requests": len(reqs), "ok": st == [0] * len(reqs)}))
        g.gace_destroy(ctx)
        return
    table, preds, samples = make_workload(args.rows, dev)
    tid = g.gace_load_columns(ctx, table.columns, borrow=True)
    if args.case.startswith("narrow"):
        cols = [0, 1, 2, 3] if args.case == "narrow_4xi32" else [0]
        pred = [[Term(c, RANGE, 0, 1000) for c in cols]]
        smp = [Sample(ROWS, 0.01, 42)] if args.case == "narrow_rows1pct" else [Sample(FULL)]
        for _ in range(3):
            g.gace_probe_batch(ctx, tid, pred, smp, table.dtypes)
    elif args.case == "wide_batch":
        for _ in range(1):
            g.gace_probe_batch(ctx, tid, preds, samples, table.dtypes, marginals=True)
    elif args.case == "hll_i32":
        for _ in range(3):
            g.gace_ndv(ctx, tid, 0, 14, 42)
    elif args.case == "materialize":
        from workloads import BLOCKS
        for smp in (Sample(ROWS, 0.01, 42), Sample(BLOCKS, 0.01, 42, 4096), Sample(ROWS, 0.1, 42)):
            sid, _ = g.gace_sample_materialize(ctx, tid, smp)
            g.gace_unload(ctx, sid)
    print(json.dumps({"case": args.case, "rows": args.rows}))
    g.gace_destroy(ctx)


def main():
    args = parse_args()
    if args.case:
        run_case(args)
        return
    d = Dist()
    if args.impl == "reference":
        run_reference(args, d)
        return
    run_gace(args, d)


if __name__ == "__main__":
    main()
