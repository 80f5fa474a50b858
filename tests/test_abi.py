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


def test_binding_struct_layouts_match_the_header():
    # every struct the binding passes by pointer: the same size and the same
    # offset for every field, from a C program built against include/spai.h
    import tempfile
    from paper_2510_27517_gb300 import spai as B
    pairs = {"spai_csr": B._CSR, "spai_gnn_weights": B._GNNW, "spai_pcg_opts": B._Opts,
             "spai_pcg_result": B._Res, "spai_schedule": B._Sched, "spai_adamw_cfg": B._AdamW,
             "spai_system_layout": B._Layout, "spai_serve_cfg": B._ServeCfg, "spai_completion": B._Completion}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "spai.h"', "int main(void) {"]
    want = []
    for cname, S in pairs.items():
        lines.append(f'  printf("%zu\\n", sizeof({cname}));')
        want.append(ctypes.sizeof(S))
        for fname, _ in S._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {fname}));')
            want.append(getattr(S, fname).offset)
    lines += ["  return 0;", "}"]
    d = tempfile.mkdtemp(prefix="abi_layout_")
    src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
    open(src, "w").write("\n".join(lines) + "\n")
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe])
    got = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    assert got == want
