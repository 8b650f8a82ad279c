"""The C-ABI library loads and exports every function that include/nlfem.h
declares (no compute call: no GPU is needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "nlfem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(nl_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


def _lib_path():
    from paper_2302_07499_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("nl_mesh_create", "nl_pairs_build", "nl_assemble", "nl_solve"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(_lib_path())
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_lists_every_declared_symbol():
    import paper_2302_07499_gb300 as nl
    assert sorted(nl.EXPORTED) == _declared()


def test_version_and_error_string_need_no_gpu():
    lib = ctypes.CDLL(_lib_path())
    lib.nl_version.restype = ctypes.c_char_p
    lib.nl_last_error.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.nl_version()
    assert isinstance(lib.nl_last_error(), bytes)
