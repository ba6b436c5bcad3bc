"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares (no compute call: this runs without a GPU)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(spamm_\w+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_header_declares_the_entry_points():
    names = _declared()
    for need in ("spamm_multiply", "spamm_truncate", "spamm_purify", "spamm_cse",
                 "spamm_mat_from_dense", "spamm_create"):
        assert need in names


def test_library_exports_every_declared_symbol():
    import paper_2005_10680_gb300 as sp
    lib = sp.load_library()
    assert os.path.dirname(sp.library_path()).startswith(ROOT)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2005_10680_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if os.path.isfile(path) and path.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            text = open(path).read()
            assert "import oracle" not in text and "from oracle" not in text, path
            assert "liboracle" not in text, path


def test_strerror_without_gpu():
    import paper_2005_10680_gb300 as sp
    lib = sp.load_library()
    assert lib.spamm_strerror(0) == b"ok"
    assert lib.spamm_strerror(1) == b"invalid argument"


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # no CPU fallback: without the built CUDA library the binding raises
    from paper_2005_10680_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "library_path", lambda: str(tmp_path / "missing.so"))
    import pytest
    with pytest.raises(ImportError):
        _lib.load_library(build_if_stale=False)


def test_context_without_gpu_raises():
    # on a machine without a GPU, creating a context is an error, not a fallback
    import pytest
    import torch

    import paper_2005_10680_gb300 as sp
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(sp.SpammError):
        sp.Context(0)
