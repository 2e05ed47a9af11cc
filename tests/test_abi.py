"""The C ABI: every function declared in include/*.h is exported by the built
library and bound by the Python layer (no GPU needed: nothing is computed)."""
import ctypes
import os
import re
import subprocess

import paper_2111_13655_gb300 as sg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(inc, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(sg_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["sg_create", "sg_apply_H", "sg_size", "sg_destroy", "sg_last_error",
                 "sg_index_map", "sg_apply_H_host", "sg_plan"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    path = sg.LIB_PATH
    if not os.path.exists(path):
        from paper_2111_13655_gb300 import build
        build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    assert declared_functions() <= exported


def test_binding_covers_every_declared_symbol():
    assert declared_functions() <= set(sg.SIGNATURES)
    sg.lib()  # loads and sets every signature


def test_last_error_without_context_is_a_string():
    assert isinstance(sg.sg_last_error(None), str)
