"""Argument checks of the Python binding (CPU only): every buffer handed to a
kernel must be a contiguous CUDA tensor of the right dtype and length, else
the call raises before anything reaches the C ABI."""
import pytest
import torch

from paper_2606_05297_gb300 import cvq


def test_dev_rejects_bad_buffers():
    ok = torch.zeros(8, dtype=torch.complex128)
    with pytest.raises(ValueError, match="dtype"):
        cvq._dev(torch.zeros(8, dtype=torch.complex64), "c128", 8, "psi")
    with pytest.raises(ValueError, match="contiguous"):
        cvq._dev(torch.zeros(16, dtype=torch.complex128)[::2], "c128", 8, "psi")
    with pytest.raises(ValueError, match="need at least 9"):
        cvq._dev(ok, "c128", 9, "psi")
    with pytest.raises(ValueError, match="CUDA"):
        cvq._dev(ok, "c128", 8, "psi")
    with pytest.raises(ValueError, match="torch tensor"):
        cvq._dev(ok.numpy(), "c128", 8, "psi")
    with pytest.raises(ValueError, match="float64"):
        cvq._dev(torch.zeros(4, dtype=torch.float32), "f64", 4, "grad")
