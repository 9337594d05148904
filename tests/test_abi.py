"""The C-ABI library loads and exports every symbol include/sophie.h declares.

No compute call is made here (no GPU is needed): only argument checks that
fail before any CUDA call.
"""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sophie.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sophie_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1301_4539_gb300 import build, sophie
    build.build()
    return sophie.load()


def test_header_declares_the_core_api():
    names = declared_functions()
    for n in ["sophie_create_grid", "sophie_set_materials", "sophie_add_source", "sophie_step",
              "sophie_read_probe", "sophie_energy", "sophie_destroy_grid"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1301_4539_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (sophie_[a-z_]+)", out))
    for n in declared_functions():
        assert n in exported, n
        assert hasattr(lib, n)


def test_binding_covers_every_symbol():
    from paper_1301_4539_gb300 import sophie
    for n in declared_functions():
        assert n in sophie.SIGNATURES, n
        assert callable(getattr(sophie, n)), n


def test_argument_errors_without_gpu(lib):
    h = ctypes.c_void_p()
    assert lib.sophie_version() == 10000
    assert lib.sophie_create_grid(0, 4, 4, 1e-3, 1e-12, ctypes.byref(h)) == -1
    assert b"sizes" in lib.sophie_last_error()
    assert lib.sophie_create_grid(4, 4, 4, -1.0, 1e-12, ctypes.byref(h)) == -1
    assert lib.sophie_create_grid(4, 4, 4, 1e-3, 0.0, ctypes.byref(h)) == -1
    # dt above the Courant limit dx / (c sqrt 3) = 1.9259e-12 s for dx = 1 mm
    assert lib.sophie_create_grid(4, 4, 4, 1e-3, 1.93e-12, ctypes.byref(h)) == -2
    assert lib.sophie_create_grid(4, 4, 4, 1e-3, 1e-12, None) == -1
    assert lib.sophie_destroy_grid(None) == 0
    assert lib.sophie_step(None, 1) == -1
    assert lib.sophie_energy(None, None) == -1
    assert lib.sophie_configure(None, 1, 0, 0, 0) == -1


def test_oracle_is_not_imported_by_the_package():
    pkg = os.path.join(ROOT, "paper_1301_4539_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "yee_oracle" not in txt, f
