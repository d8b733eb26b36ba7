"""The rank pass's search structures, built by the planner and searched as
the rank pass reads them, on the CPU (no GPU): tests/rank_index_check.cu
builds each coded column's level-order search tree and bucket index
(build_rank_tree, build_rank_buckets under every rank_search setting) for
random endpoint sets of 32- and 64-bit keys, emulates the kernel's searches
and compares every rank with the number of endpoints <= the key."""
import os
import shutil
import subprocess

import pytest

from conftest import ROOT


def test_rank_tree_and_bucket_index_give_every_rank(g, tmp_path):
    from paper_2512_19750_gb300 import build as b

    nvcc = os.path.join(b.cuda_home(), "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc")
    if not nvcc:
        pytest.skip("nvcc is not installed")
    exe = str(tmp_path / "rank_index_check")
    lib_dir = os.path.dirname(g._capi.LIB_PATH)
    cmd = [nvcc, "-O2", "-std=c++17", "-x", "cu", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(lib_dir, "csrc"), "-o", exe, os.path.join(ROOT, "tests", "rank_index_check.cu"),
           "-L", lib_dir, "-lgace", "-Xlinker", "-rpath," + lib_dir]
    subprocess.run(cmd, check=True, capture_output=True, timeout=600)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout + out.stderr
