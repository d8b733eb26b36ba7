"""Host parts of the library checked on the CPU (no GPU), each by a small
program built against the library: the rank pass's search structures, built
by the planner and searched as the rank pass reads them (tests/rank_index_check.cu
builds each coded column's level-order search tree and bucket index
(build_rank_tree, build_rank_buckets under every rank_search setting) for
random endpoint sets of 32- and 64-bit keys, emulates the kernel's searches
and compares every rank with the number of endpoints <= the key), the
context's host worker pool (tests/host_pool_check.cu), the batched form's
fusion rules (tests/fusion_rules_check.cu) and the probe planner's passes
(tests/plan_check.cu)."""
import os
import shutil
import subprocess

import pytest

from conftest import ROOT


def _run_host_check(g, tmp_path, name, *args):
    """Compiles tests/<name>.cu against the library's host headers, links it
    with the built library and runs it; its last line must start with "ok"."""
    from paper_2512_19750_gb300 import build as b

    nvcc = os.path.join(b.cuda_home(), "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc")
    if not nvcc:
        pytest.skip("nvcc is not installed")
    exe = str(tmp_path / name)
    lib_dir = os.path.dirname(g._capi.LIB_PATH)
    cmd = [nvcc, "-O2", "-std=c++17", "-x", "cu", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(lib_dir, "csrc"), "-o", exe, os.path.join(ROOT, "tests", name + ".cu"),
           "-L", lib_dir, "-lgace", "-Xlinker", "-rpath," + lib_dir]
    subprocess.run(cmd, check=True, capture_output=True, timeout=600)
    out = subprocess.run([exe, *args], capture_output=True, text=True, timeout=300)
    lines = out.stdout.strip().splitlines()
    assert out.returncode == 0 and lines and lines[-1].startswith("ok"), out.stdout + out.stderr


def test_rank_tree_and_bucket_index_give_every_rank(g, tmp_path):
    _run_host_check(g, tmp_path, "rank_index_check")


def test_host_worker_pool_handles_every_index_once(g, tmp_path):
    """The workers that plan and assemble a large batch (HostPool): every
    index of every run handled exactly once, over 300 runs in a row."""
    _run_host_check(g, tmp_path, "host_pool_check")


def test_fusion_rules_of_the_batched_form(g, tmp_path):
    """Which probe requests may fuse, and with which group, under each of the
    batched form's fusion rules, and the limits every rule keeps."""
    _run_host_check(g, tmp_path, "fusion_rules_check")


def test_planner_settles_every_predicate(g, tmp_path):
    """The probe planner on a seeded 1024-predicate batch of the benchmark's
    shape (1-4 terms over four int32, two int64 and two float32 columns, five
    row sets): at 100M rows (rank-coded) and at 1000 rows (not coded) every
    predicate is settled exactly once, each pass holds its predicates' terms
    within the kernel's limits, and every rank code's keys are sorted."""
    import numpy as np

    from workloads import Sample, make_predicates, make_skew_corr

    t = make_skew_corr(n=200_000, seed=1002, device="cpu")
    preds = make_predicates(t, 1024, 1, 4, seed=2002)
    batch = g.TermBatch(preds, t.dtypes)
    samples = g._samples([Sample(0), Sample(1, 0.001, 42), Sample(1, 0.01, 42), Sample(1, 0.1, 42),
                          Sample(2, 0.01, 42, 4096)])
    (tmp_path / "terms.bin").write_bytes(bytes(batch.terms))
    (tmp_path / "preds.bin").write_bytes(bytes(batch.preds))
    (tmp_path / "ins.bin").write_bytes(bytes(batch.in_values))
    (tmp_path / "samples.bin").write_bytes(bytes(samples))
    (tmp_path / "dtypes.bin").write_bytes(np.asarray(t.dtypes, dtype=np.int32).tobytes())
    _run_host_check(g, tmp_path, "plan_check", str(tmp_path))
