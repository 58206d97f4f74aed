"""The C-ABI library builds for sm_103a and exports every function declared
in include/fifa.h (no GPU needed: only loading and symbol lookup)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fifa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(fifa_[a-z_0-9A-Z]+)\s*\(", src))
    return sorted(n for n in names if not n.isupper())


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_library_exports_all_declared_symbols():
    from paper_2006_06537_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert len(declared_functions()) >= 20


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2006_06537_gb300 import fifa

    monkeypatch.setattr(fifa, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(fifa, "_lib", None)
    with pytest.raises(RuntimeError):
        fifa.lib()
