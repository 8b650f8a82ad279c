"""The product path has no CPU fallback: without the built library, or
without a CUDA device, the binding raises instead of computing anything."""
import pytest

torch = pytest.importorskip("torch")


def test_missing_library_raises(tmp_path, monkeypatch):
    from paper_2302_07499_gb300 import _binding as B
    monkeypatch.setattr(B, "LIB_PATH", str(tmp_path / "libnlfem.so"))
    monkeypatch.setattr(B, "_lib", None)
    with pytest.raises(ImportError, match="not built"):
        B.lib()


@pytest.mark.skipif(torch.cuda.is_available(), reason="a CUDA device is present")
def test_no_device_raises():
    import paper_2302_07499_gb300 as nl
    with pytest.raises((RuntimeError, AssertionError)):
        nl.Device()


@pytest.mark.skipif(torch.cuda.is_available(), reason="a CUDA device is present")
def test_c_abi_answers_no_device():
    """The library itself refuses valid work when no CUDA device exists: it
    returns NL_ECUDA with a message and leaves no handle behind."""
    import ctypes
    import numpy as np
    import nl_inputs as I
    from paper_2302_07499_gb300 import _binding as B
    L = B.lib()
    mesh, _ = I.cube_problem(2, 1)
    verts = np.ascontiguousarray(mesh.verts, dtype=np.float64)
    tets = np.ascontiguousarray(mesh.tets, dtype=np.int32)
    om = np.ascontiguousarray(mesh.tet_in_omega, dtype=np.uint8)
    nf = np.ascontiguousarray(mesh.node_free, dtype=np.uint8)
    out = ctypes.c_void_p()
    st = L.nl_mesh_create(None, verts.ctypes.data, mesh.nv, tets.ctypes.data, mesh.nt, om.ctypes.data,
                          nf.ctypes.data, B.HOST, ctypes.byref(out))
    assert st == B.NL_ECUDA and out.value is None
    assert "no CUDA device" in L.nl_last_error().decode()
    o = B.nl_server_opts(budget_bytes=10 ** 9, workers=1, queue_capacity=4, cache=0)
    assert L.nl_server_create(ctypes.byref(o), ctypes.byref(out)) == B.NL_ECUDA and out.value is None
