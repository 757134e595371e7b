"""The C library loads without a GPU and exports every symbol include/stab.h declares."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(stab_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_core_entry_points():
    names = declared_functions()
    for core in ("stab_create", "stab_apply_circuit", "stab_get_generators", "stab_expect",
                 "stab_grad", "stab_destroy"):
        assert core in names


def test_library_exports_every_declared_symbol():
    from paper_2502_10685_gb300 import _lib
    L = _lib.load()
    missing = [n for n in sorted(declared_functions()) if not hasattr(L, n)]
    assert not missing, missing


def test_host_only_calls():
    from paper_2502_10685_gb300 import _lib, stab
    L = _lib.load()
    assert L.stab_version() == 1
    assert L.stab_error_string(-5) == b"non-finite angle or coefficient"
    o = stab.stab_default_opts()
    assert o.device == -1 and o.fuse == 1 and o.kernel == 0
