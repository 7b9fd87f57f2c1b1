"""CPU checks of the C-ABI boundary: the library loads without a GPU and exports
every entry point include/*.h declares; the binding knows every one of them."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(mm_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1501_07293_b300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("mm_create", "mm_destroy", "mm_set_m", "mm_get_m", "mm_set_field", "mm_heff", "mm_step",
              "mm_energy", "mm_observables", "mm_last_error"):
        assert n in names, n


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in sorted(_declared()) if not hasattr(L, n)]
    assert not missing, missing


def test_exports_are_c_symbols(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    for n in _declared():
        assert n in exported, n   # unmangled, i.e. extern "C"


def test_binding_covers_every_declared_symbol(libpath):
    from paper_1501_07293_b300 import solver
    assert _declared() <= set(solver._SIGNATURES), _declared() - set(solver._SIGNATURES)
    solver.lib()   # loads and sets every signature


def test_no_cpu_fallback_in_the_product_path():
    # the package never imports the oracle
    for f in glob.glob(os.path.join(ROOT, "paper_1501_07293_b300", "*.py")):
        src = open(f).read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), f
        assert "importlib" not in src, f


def test_create_without_gpu_fails_cleanly(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = ctypes.CDLL(libpath)
    L.mm_create.restype = ctypes.c_int
    L.mm_last_error.restype = ctypes.c_char_p
    ctx = ctypes.c_void_p()
    g = (ctypes.c_int * 3)(8, 4, 1)
    d = ctypes.c_double
    rc = L.mm_create(ctypes.byref(ctx), g, d(4e-9), d(8e5), d(1.3e-11), d(0.0), d(0.02), d(1.76e11), None)
    assert rc != 0 and not ctx.value
    assert L.mm_last_error(None)


def test_bounds_check_build_exports_the_same_boundary():
    from paper_1501_07293_b300 import build
    path = build.build(bounds_check=True)
    L = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared()) if not hasattr(L, n)]
    assert not missing, missing
    L.mm_build_flags.restype = ctypes.c_int
    assert L.mm_build_flags() & 1
    L2 = ctypes.CDLL(build.build())
    L2.mm_build_flags.restype = ctypes.c_int
    assert L2.mm_build_flags() == 0
