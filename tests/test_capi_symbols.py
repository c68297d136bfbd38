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


def test_binding_holds_no_method_arithmetic():
    """The Python layer only marshals: the binding and the learned-guess driver contain no matrix products
    and no numerical functions applied to the method's data (Fock assembly, density blocks, learning-rate
    schedules and training steps all run in the library).  Checked on their syntax trees."""
    import ast
    import paper_1708_00033_gb300 as pkg
    root = os.path.dirname(pkg.__file__)
    banned_calls = {"cos", "sin", "exp", "log", "sqrt", "einsum", "dot", "matmul", "tensordot", "trace", "outer",
                    "eigh", "solve", "cholesky", "inv", "tanh"}
    for name in ("hf.py", "guess.py"):
        tree = ast.parse(open(os.path.join(root, name)).read())
        for node in ast.walk(tree):
            assert not (isinstance(node, ast.BinOp) and isinstance(node.op, ast.MatMult)), (name, node.lineno)
            if isinstance(node, ast.Call) and isinstance(node.func, ast.Attribute):
                f = node.func
                base = f.value.id if isinstance(f.value, ast.Name) else (
                    f.value.attr if isinstance(f.value, ast.Attribute) else "")
                if base in ("np", "numpy", "math", "torch", "linalg"):
                    assert f.attr not in banned_calls, (name, node.lineno, f.attr)
            # no arithmetic that combines two matrices (X + Y, X - c * Y, ...): binary +/-/* whose operands
            # are both names, subscripts or calls
            if isinstance(node, ast.BinOp) and isinstance(node.op, (ast.Add, ast.Sub, ast.Mult)):
                kinds = (ast.Name, ast.Subscript, ast.Call, ast.BinOp)
                if isinstance(node.left, kinds) and isinstance(node.right, kinds):
                    names = {n.id for n in ast.walk(node) if isinstance(n, ast.Name)}
                    assert not names & {"H", "J", "K", "F", "P", "S", "C"}, (name, node.lineno)


def test_binding_constants_match_header():
    """Every HF_* integer constant of the binding equals the header's #define of that name, and every flag
    and status code the header defines exists in the binding."""
    import re
    from paper_1708_00033_gb300 import hf
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    txt = open(os.path.join(root, "include", "hf.h")).read()
    defs = {m.group(1): int(m.group(2)) for m in re.finditer(r"^#define (HF_\w+)\s+(-?\d+)\b", txt, re.M)}
    assert defs["HF_OBARA_SAIKA"] == 64 and defs["HF_RYS"] == 32
    for name, value in vars(hf).items():
        if name.startswith("HF_") and isinstance(value, int) and name in defs:
            assert value == defs[name], name
    for name in defs:
        if name.startswith(("HF_E_", "HF_PTR_")) or name in ("HF_OK", "HF_TIMING", "HF_FP64_ONLY", "HF_DENSITY_SCREEN",
                                                              "HF_RYS", "HF_OBARA_SAIKA", "HF_SP_SHELL",
                                                              "HF_BATCH_SEQUENTIAL"):
            assert getattr(hf, name) == defs[name], name
    assert hf.NUM_CLASSES == defs["HF_NUM_CLASSES"]
