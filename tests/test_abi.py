"""The C ABI: the library builds for sm_103a, loads, and exports every
function include/spai.h declares; the Python binding binds exactly those.
No compute call is made here (no GPU needed)."""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "spai.h")


def declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*(spai_[a-z_0-9]+)\s*\(", txt, flags=re.M)))


def test_header_declares_the_boundary_calls():
    names = declared()
    for must in ("spai_build_pattern", "spai_gnn_precond", "spai_pcg_solve", "spai_pcg_solve_batched",
                 "spai_server_create", "spai_server_submit", "spai_server_poll", "spai_server_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2510_27517_gb300 import _build
    lib_path = _build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (spai_\w+)", out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing
    L = ctypes.CDLL(lib_path)
    for n in declared():
        assert getattr(L, n) is not None


def test_binding_matches_header():
    from paper_2510_27517_gb300 import spai
    assert sorted(spai.exported_symbols()) == declared()


def test_version_and_error_strings_without_gpu():
    from paper_2510_27517_gb300 import _build
    L = ctypes.CDLL(_build.build())
    L.spai_version.restype = ctypes.c_char_p
    L.spai_last_error.restype = ctypes.c_char_p
    assert b"sm_103a" in L.spai_version()
    # a null-argument call fails cleanly before touching the device
    L.spai_build_pattern.restype = ctypes.c_int
    assert L.spai_build_pattern(None, 0, None, None) == -1
    assert L.spai_last_error()
