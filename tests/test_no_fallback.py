"""The product path has no CPU fallback: without its CUDA library the binding
raises, and host (CPU) tensors are refused rather than computed on the host.
CPU only."""
import pytest
import torch

from paper_2103_10329_gb300 import mgct


def test_missing_library_raises(monkeypatch, tmp_path):
    monkeypatch.setattr(mgct, "_lib", None)
    monkeypatch.setattr(mgct, "LIB_PATH", str(tmp_path / "libmgct.so"))
    with pytest.raises(mgct.MgctError, match="missing"):
        mgct.lib()


def test_host_tensors_are_refused():
    from paper_2103_10329_gb300 import build
    build.build()
    x = torch.zeros((8, 8, 8))
    with pytest.raises(mgct.MgctError, match="CUDA tensor"):
        mgct.restrict_volume(x, out=torch.zeros((4, 4, 4)))
    with pytest.raises(mgct.MgctError, match="CUDA tensor"):
        mgct.prolong_add(torch.zeros((4, 4, 4)), torch.zeros((4, 4, 4)), x)
