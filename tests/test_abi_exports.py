"""The C ABI library builds for sm_103a and exports every entry point that
include/apo.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "apo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(apo_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("apo_hash_tasks", "apo_find_repeats", "apo_match_candidates", "apo_create",
              "apo_destroy", "apo_last_error"):
        assert s in syms


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_library_exports_every_declared_symbol():
    from paper_2406_18111_gb300 import build as b
    path = b.build()
    lib = ctypes.CDLL(path)
    for s in declared_symbols():
        assert hasattr(lib, s), s
    import paper_2406_18111_gb300 as P
    assert set(P.EXPORTS) == set(declared_symbols())
    # every entry point has its argument types declared: ctypes would
    # otherwise pass a Python int (a host pointer, a 64-bit size) as a C int
    L = P.lib()
    for s in P.EXPORTS:
        assert getattr(L, s).argtypes is not None, s


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2406_18111_gb300 as P
    monkeypatch.setattr(P, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(P, "_lib", None)
    with pytest.raises(RuntimeError):
        P.lib()
