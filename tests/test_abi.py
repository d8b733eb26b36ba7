"""The C-ABI library loads without a GPU and exports every function that
include/gace.h declares (no compute calls here)."""
import os
import re

from conftest import ROOT


def _declared():
    with open(os.path.join(ROOT, "include", "gace.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gace_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("gace_create", "gace_destroy", "gace_load_columns", "gace_unload", "gace_probe_batch",
              "gace_ndv", "gace_join_card", "gace_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(g):
    import ctypes

    lib = ctypes.CDLL(g._capi.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(_declared()) == set(g._capi.PROTOTYPES), "binding prototypes differ from the header"


def test_abi_version_and_status_names(g):
    assert g.gace_abi_version() == 4
    assert g.gace_status_string(0) == "GACE_OK"
    assert g.gace_status_string(7) == "GACE_EOVERFLOW"
    assert g.gace_status_string(99) == "GACE_UNKNOWN"


def test_oracle_is_not_reachable_from_the_product():
    """The product package neither imports nor links the oracle."""
    pkg = os.path.join(ROOT, "paper_2512_19750_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                with open(os.path.join(dirpath, fn)) as f:
                    src = f.read()
                assert "oracle" not in src.lower().replace("the oracle", ""), fn
                assert "orc_" not in src, fn
