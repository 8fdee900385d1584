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


def test_argument_checks_answer_without_a_gpu():
    """Entry points reject bad arguments before touching the device."""
    import ctypes as C
    from paper_2604_12505_gb300 import build
    from paper_2604_12505_gb300._lib import SphParams
    lib = C.CDLL(build.build())
    n = C.c_int32()
    for nx, want in ((2, 2 * 25 + 20 + 29), (4, 155), (6, 2 * 81 + 36 + 29), (8, 315)):
        assert lib.slpv_n_params(nx, C.byref(n)) == 0 and n.value == want
    assert lib.slpv_n_params(3, C.byref(n)) == -1
    out = C.c_void_p()
    assert lib.slpv_create(None, C.byref(out)) == -1
    p = SphParams(dx=0.01, h_over_dx=1.3, n_rings=0)
    g = C.c_double()
    assert lib.sph_gamma1_estimate(C.byref(p), C.byref(g)) == -1
    assert lib.sph_gamma1_estimate(None, C.byref(g)) == -1
    # the no-allocation density call rejects sizes beyond its fixed array
    # before any device work (host buffers stand in for the device pointers
    # and are never dereferenced)
    lib.sph_density_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p,
                                        C.c_void_p, C.c_void_p]
    lib.sph_last_error.restype = C.c_char_p
    q = SphParams(R=0.5, dx=0.02, h_over_dx=1.3, n_rings=3, rho0=1000.0)
    buf = (C.c_double * 8)()
    ptr = C.cast(buf, C.c_void_p)
    assert lib.sph_density_noalloc(C.byref(q), ptr, 4, ptr, 16385, ptr, ptr, None) == -6
    assert b"16384" in lib.sph_last_error()
    assert lib.sph_density_noalloc(C.byref(q), ptr, -1, ptr, 0, ptr, ptr, None) == -1
    assert lib.sph_density_noalloc(C.byref(q), None, 4, ptr, 0, ptr, ptr, None) == -1
