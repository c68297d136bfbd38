"""The C-ABI library loads and exports every entry point include/hf.h declares."""
import ctypes
import os

import pytest


def test_header_declares_entry_points():
    from paper_1708_00033_gb300 import hf
    names = hf.exported_symbols()
    for must in ("hf_create", "hf_destroy", "hf_system_create", "hf_fock_build", "hf_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1708_00033_gb300 import hf
    if not os.path.exists(hf.LIB_PATH):
        import paper_1708_00033_gb300 as pkg
        pkg.build()
    lib = ctypes.CDLL(hf.LIB_PATH)
    missing = [n for n in hf.exported_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    from paper_1708_00033_gb300 import hf
    lib = hf.load_library()
    for code in (0, -1, -2, -3, -4, -5, -6, 17):
        assert lib.hf_strerror(code)


def test_no_device_is_reported_not_crashed():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1708_00033_gb300 import hf
    lib = hf.load_library()
    h = ctypes.c_void_p()
    rc = lib.hf_create(ctypes.byref(h), 0, None)
    assert rc in (hf.HF_E_UNSUPPORTED, hf.HF_E_CUDA, hf.HF_E_INVALID)
    assert not h.value


def test_missing_library_fails_loudly(monkeypatch):
    """No fallback: without the built CUDA library the binding raises."""
    from paper_1708_00033_gb300 import hf
    monkeypatch.setattr(hf, "_lib", None)
    monkeypatch.setattr(hf, "LIB_PATH", os.path.join(os.path.dirname(hf.LIB_PATH), "does-not-exist.so"))
    with pytest.raises(RuntimeError):
        hf.load_library()


def test_product_does_not_use_the_oracle():
    """The package (binding, drivers, CUDA sources) never imports or links the oracle."""
    import re
    import paper_1708_00033_gb300 as pkg
    root = os.path.dirname(pkg.__file__)
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle|#include\s+[\"<].*oracle)", re.M)
    hits = []
    for d, _, files in os.walk(root):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                with open(os.path.join(d, f)) as fh:
                    if pat.search(fh.read()):
                        hits.append(f)
    assert not hits, hits
