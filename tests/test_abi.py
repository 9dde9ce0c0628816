"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/fhecnn.h declares; the binding refuses to run without it."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fhecnn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fhe_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("fhe_ctx_create", "fhe_keygen", "fhe_encode", "fhe_encrypt", "fhe_decrypt", "fhe_decode",
                 "fhe_eval_conv", "fhe_eval_quad_act", "fhe_eval_pool_dense", "fhe_rescale", "fhe_rotate",
                 "fhe_infer", "fhe_ct_export", "fhe_ct_import", "fhe_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2509_22857_gb300 import build
    path = build.build()
    so = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(so, n)]
    assert not missing, missing
    from paper_2509_22857_gb300 import _lib
    assert set(_lib.EXPORTED) <= set(_declared())


def test_binding_fails_loudly_without_library(monkeypatch):
    from paper_2509_22857_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", "/nonexistent/libfhecnn.so")
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.lib()


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2509_22857_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", text).lower(), f


def test_binding_error_codes_match_the_header():
    from paper_2509_22857_gb300 import _lib
    src = open(os.path.join(ROOT, "include", "fhecnn.h")).read()
    codes = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(FHE_(?:OK|E_[A-Z]+))\s+(-?\d+)", src)}
    assert set(codes) == {"FHE_OK", "FHE_E_INVAL", "FHE_E_LEVEL", "FHE_E_NOKEY", "FHE_E_OOM", "FHE_E_CUDA",
                          "FHE_E_TIMEOUT"}
    for name, v in codes.items():
        assert getattr(_lib, name) == v, name
