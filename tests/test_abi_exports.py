"""The C-ABI library loads and exports every function its headers declare.

CPU only: loading the library and resolving symbols needs no GPU; no compute
entry point is called here.
"""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z_0-9]*\s*\**\s*\**\s*([A-Za-z_][A-Za-z_0-9]*)\s*\(",
                             src, flags=re.M):
            if m.group(1) not in ("if", "while", "for", "return", "sizeof"):
                names.append(m.group(1))
    return sorted(set(names))


def test_headers_declare_entry_points():
    names = declared_functions()
    for must in ("pr_create", "pr_destroy", "pr_props", "pr_T_from_h", "pr_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(prlib):
    missing = [n for n in declared_functions() if not hasattr(prlib, n)]
    assert not missing, missing


def test_version_and_error_string_without_gpu(prlib):
    prlib.pr_version.restype = ctypes.c_char_p
    assert b"sm_103a" in prlib.pr_version()
    prlib.pr_last_error.restype = ctypes.c_char_p
    assert isinstance(prlib.pr_last_error(), bytes)


def test_host_validation_rejects_bad_arguments(prlib):
    """Argument checks run on the host before any CUDA call."""
    vp = ctypes.c_void_p
    prlib.pr_create.argtypes = [vp, ctypes.POINTER(vp)]
    out = vp()
    assert prlib.pr_create(None, ctypes.byref(out)) == -1
    prlib.pr_props.argtypes = [vp, ctypes.c_int, ctypes.c_int64] + [vp] * 3 + [ctypes.c_int64] + [vp] * 8
    assert prlib.pr_props(None, 0, 10, *([None] * 3), 10, *([None] * 8)) == -1
