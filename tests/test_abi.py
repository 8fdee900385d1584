"""The C-ABI library loads and exports every symbol its headers declare
(no compute: runs without a GPU)."""
import ctypes
import glob
import os
import re

from tests.conftest import ROOT


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([a-z][a-z0-9_]*)\s*\(", src, re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2604_12505_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert {"sph_create", "sph_step", "sph_run_batch", "sph_eval"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_raises_without_gpu_or_library(monkeypatch):
    import pytest
    torch = pytest.importorskip("torch")
    from paper_2604_12505_gb300 import sph
    if not torch.cuda.is_available():
        with pytest.raises(RuntimeError):
            sph.Sim({})
    from paper_2604_12505_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", "/nonexistent/libgb300sloshing.so")
    with pytest.raises(ImportError):
        _lib.lib()
