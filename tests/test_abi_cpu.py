"""Host-side checks of the C interface (no GPU): the library builds for sm_103a, loads, and
exports every entry point that include/fc4.h declares; the binding refuses to run without it."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2510_00518_gb300 import build as fc4_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fc4_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    return fc4_build.build()


def test_header_declares_the_interface():
    names = declared_symbols()
    for n in ("fc4_init", "fc4_rates", "fc4_kappa", "fc4_rates_backward", "fc4_processes",
              "fc4_set_modes", "fc4_update_anharmonic", "fc4_last_error", "fc4_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for n in declared_symbols():
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (fc4_\w+)", out))
    assert set(declared_symbols()) <= exported


def test_build_targets_sm103a_only():
    assert fc4_build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_last_error_without_gpu_calls(libpath):
    lib = ctypes.CDLL(libpath)
    lib.fc4_last_error.restype = ctypes.c_char_p
    lib.fc4_last_error.argtypes = [ctypes.c_void_p]
    assert isinstance(lib.fc4_last_error(None), bytes)
    # fc4_init rejects a NULL output pointer before touching the device
    lib.fc4_init.restype = ctypes.c_int
    assert lib.fc4_init(None, None, None, None, None, None, None) == 1


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_2510_00518_gb300 as pkg
    monkeypatch.setattr(pkg, "_LIB", None)
    monkeypatch.setattr(pkg._build, "LIB", str(tmp_path / "missing" / "libfc4.so"))
    with pytest.raises(ImportError):
        pkg.load()
