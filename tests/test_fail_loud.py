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
