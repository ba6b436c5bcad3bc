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


def test_entry_points_reject_null_handles_without_a_gpu():
    """Every entry point checks its handles before any CUDA call: null handles give
    SPAMM_EINVAL (1) with a message, the query calls give their documented neutral
    answers, and the release calls are no-ops."""
    import paper_2005_10680_gb300 as sp
    lib = sp.load_library()
    null = None
    calls = {
        "spamm_create": lambda: lib.spamm_create(null, 0, null),
        "spamm_set_bound": lambda: lib.spamm_set_bound(null, 0),
        "spamm_set_tau_table": lambda: lib.spamm_set_tau_table(null, 1.0, 0.9),
        "spamm_mat_from_dense": lambda: lib.spamm_mat_from_dense(null, null, 64, 64, 64, 0.0, 0, null),
        "spamm_mat_from_blocks": lambda: lib.spamm_mat_from_blocks(null, 64, 64, 0, null, null, null, 0,
                                                                   null),
        "spamm_mat_to_dense": lambda: lib.spamm_mat_to_dense(null, null, null, 64, 0),
        "spamm_mat_to_blocks": lambda: lib.spamm_mat_to_blocks(null, null, null, null, null, 0),
        "spamm_mat_get_blocks": lambda: lib.spamm_mat_get_blocks(null, null, 1, null, null, null,
                                                                  null),
        "spamm_mat_info": lambda: lib.spamm_mat_info(null, null, null, null),
        "spamm_mat_block_norms": lambda: lib.spamm_mat_block_norms(null, null, null),
        "spamm_mat_block_map": lambda: lib.spamm_mat_block_map(null, null, null),
        "spamm_cse": lambda: lib.spamm_cse(null, null, null, null, 0, null),
        "spamm_multiply": lambda: lib.spamm_multiply(null, null, null, 1e-6, 0, null, null),
        "spamm_multiply_tau": lambda: lib.spamm_multiply_tau(null, null, null, 0.0, 0, null, null),
        "spamm_sp2_step": lambda: lib.spamm_sp2_step(null, null, 0, 1e-6, 0.0, 0, null, null),
        "spamm_truncate": lambda: lib.spamm_truncate(null, null, 1e-6, 1, null),
        "spamm_purify": lambda: lib.spamm_purify(null, null, 1, 1e-5, 10, null, null, null),
        "spamm_purify_batched": lambda: lib.spamm_purify_batched(null, 0, null, null, 1e-5, 10, null, 1,
                                                                 null, null, null),
        "spamm_autotune": lambda: lib.spamm_autotune(null, null, 1e-6, 1, null),
        "spamm_cse_search_noalloc": lambda: lib.spamm_cse_search_noalloc(null, null, 8, 1e-6, null, null,
                                                                         null, null),
    }
    for name, call in calls.items():
        assert call() == 1, name
        assert lib.spamm_last_error(), name
    assert lib.spamm_prec_supported(null, 0, 64) == 0
    assert lib.spamm_ctx_launches(null) == 0
    lib.spamm_destroy(null)
    lib.spamm_mat_free(null)
    assert lib.spamm_debug_fail_alloc(-1) == 0          # the test hook needs no GPU either


def test_header_is_c_and_the_library_links_from_c(tmp_path):
    """include/spamm.h compiles as strict C99 and a C program links against the
    library and calls it (an argument error needs no GPU)."""
    import shutil
    import subprocess

    import paper_2005_10680_gb300 as sp
    if shutil.which("gcc") is None:
        import pytest
        pytest.skip("no C compiler")
    lib = sp.library_path()
    src = tmp_path / "use_spamm.c"
    src.write_text(
        "#include <stdio.h>\n#include \"spamm.h\"\n"
        "int main(void) {\n"
        "    spamm_ctx* ctx = NULL;\n"
        "    spamm_mat* m = NULL;\n"
        "    spamm_report rep;\n"
        "    spamm_purify_opts opts;\n"
        "    (void)rep; (void)opts; (void)m;\n"
        "    int st = spamm_create(NULL, 0, NULL);\n"
        "    if (st != SPAMM_EINVAL) return 1;\n"
        "    st = spamm_multiply(ctx, NULL, NULL, 1e-6, SPAMM_MIXED, &m, NULL);\n"
        "    if (st != SPAMM_EINVAL) return 2;\n"
        "    printf(\"%s\\n\", spamm_last_error());\n"
        "    return 0;\n"
        "}\n")
    exe = tmp_path / "use_spamm"
    libdir = os.path.dirname(lib)
    name = os.path.basename(lib)[3:-3]                    # libNAME.so -> NAME
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                           "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir,
                           "-l" + name, "-Wl,-rpath," + libdir, "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out
    assert "spamm_multiply" in out.stdout
