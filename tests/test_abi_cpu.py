"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and exports every
function declared in include/peps_gb300.h (no compute call: there is no GPU here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", txt, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "defined")))


def test_header_declares_the_abi():
    names = _declared()
    for n in ("peps_create", "peps_destroy", "peps_set_params", "peps_amplitudes", "peps_local_energy",
              "peps_logderiv", "peps_evaluate", "minsr_step", "peps_sample"):
        assert n in names


def test_library_builds_loads_and_exports_every_declared_symbol():
    from paper_2503_12557_gb300 import build, peps
    path = build.build()
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert hasattr(lib, n), n
    assert set(peps.exported_symbols()) <= set(_declared())


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2503_12557_gb300 import peps
    monkeypatch.setattr(peps, "_LIB", None)
    monkeypatch.setattr(peps, "_LIBPATH", str(tmp_path / "missing.so"))
    try:
        peps.load()
    except RuntimeError as e:
        assert "not built" in str(e)
    else:
        raise AssertionError("load() must raise when the library is missing")
