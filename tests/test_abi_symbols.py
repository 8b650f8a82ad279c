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


def test_argument_errors_need_no_gpu():
    """Each entry point checks its arguments before any device work and
    answers NL_EINVAL with a message (the header's error contract)."""
    from paper_2302_07499_gb300 import _binding as B
    L = B.lib()
    out = ctypes.c_void_p()
    msg = lambda: L.nl_last_error().decode()

    assert L.nl_server_create(None, ctypes.byref(out)) == B.NL_EINVAL and out.value is None
    for bad in (dict(workers=0), dict(workers=17), dict(budget_bytes=0), dict(queue_capacity=0)):
        o = B.nl_server_opts(**dict(dict(budget_bytes=10 ** 9, workers=1, queue_capacity=4, cache=0), **bad))
        assert L.nl_server_create(ctypes.byref(o), ctypes.byref(out)) == B.NL_EINVAL, bad
        assert "workers 1..16" in msg()
    t = ctypes.c_uint64()
    assert L.nl_server_submit(None, None, ctypes.byref(t)) == B.NL_EINVAL and msg() == "NULL argument"
    assert L.nl_server_poll(None, 1, None) == B.NL_EINVAL
    assert L.nl_server_release(None, 1) == B.NL_EINVAL
    assert L.nl_batch_system(None, 0, ctypes.byref(out)) == B.NL_EINVAL
    assert L.nl_batch_get_info(None, None) == B.NL_EINVAL
    assert L.nl_pairs_build(None, 0.1, ctypes.byref(out)) == B.NL_EINVAL and msg() == "NULL argument"
    assert L.nl_assemble(None, None, ctypes.byref(out)) == B.NL_EINVAL
    for cells, lo, hi in ((0, 0.0, 1.0), (1001, 0.0, 1.0), (4, 1.0, 1.0), (4, float("nan"), 1.0)):
        assert L.nl_mesh_create_box(None, lo, hi, cells, 0.0, 1.0, 0.0, 0, ctypes.byref(out)) == B.NL_EINVAL
        assert "bad box" in msg() and out.value is None
    for jit in (-0.1, 0.5, float("nan")):
        assert L.nl_mesh_create_box(None, -0.25, 1.25, 6, 0.0, 1.0, jit, 7, ctypes.byref(out)) == B.NL_EINVAL
        assert "jitter_frac" in msg() and out.value is None
    assert L.nl_probe_philox(None, 0, 4, None) == B.NL_EINVAL
    # a later successful call clears the message
    assert L.nl_probe_philox(ctypes.c_void_p(1), 0, 0, ctypes.c_void_p(1)) == B.NL_OK and msg() == ""
