"""Repository rules that need no GPU: nothing committed reaches into the
scratch folder, and every profile summary is short text that names the
command it came from."""
import os
import re

from conftest import ROOT


def _sources():
    for top in ("paper_2512_19750_gb300", "tests", "workloads", "oracle"):
        for dirpath, _, files in os.walk(os.path.join(ROOT, top)):
            for fn in files:
                if fn.endswith((".py", ".cu", ".cuh", ".cpp", ".h", ".c")):
                    yield os.path.join(dirpath, fn)
    for fn in ("bench.py", "__graft_entry__.py"):
        yield os.path.join(ROOT, fn)


def test_nothing_committed_uses_the_scratch_folder():
    pat = re.compile(r"""["'/]_work[/"']""")
    for path in _sources():
        if os.path.basename(path) == "test_repo_rules.py":
            continue
        with open(path, errors="replace") as f:
            assert not pat.search(f.read()), path


def test_profiles_are_short_text_with_their_command():
    d = os.path.join(ROOT, "profiles")
    for fn in os.listdir(d):
        path = os.path.join(d, fn)
        assert fn.endswith((".md", ".txt", ".json")), fn
        assert os.path.getsize(path) < 16 * 1024, fn
        if fn.endswith(".md"):
            with open(path) as f:
                text = f.read()
            assert "Command" in text and ("ncu " in text or "bench.py" in text), fn
