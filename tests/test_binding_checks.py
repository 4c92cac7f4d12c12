"""Argument checks of the ctypes binding that need no GPU: device buffers are
validated before their raw pointer reaches the library."""
import pytest
import torch

import paper_2606_30985_gb300 as pkg


def test_device_tensor_rejects_host_wrong_dtype_short_and_strided():
    with pytest.raises(pkg.PepoError, match="GPU"):
        pkg._device_tensor(torch.zeros(16, dtype=torch.uint8), torch.uint8, 8, "save_state")
    with pytest.raises(pkg.PepoError, match="torch tensor"):
        pkg._device_tensor(b"\x00" * 16, torch.uint8, 8, "save_state")


@pytest.mark.gpu
def test_device_tensor_checks_on_cuda():
    t = torch.zeros(16, dtype=torch.uint8, device="cuda")
    assert pkg._device_tensor(t, torch.uint8, 16, "x") is t
    with pytest.raises(pkg.PepoError, match="dtype"):
        pkg._device_tensor(t, torch.float32, 1, "x")
    with pytest.raises(pkg.PepoError, match="at least"):
        pkg._device_tensor(t, torch.uint8, 17, "x")
    with pytest.raises(pkg.PepoError, match="contiguous"):
        pkg._device_tensor(torch.zeros(4, 4, dtype=torch.uint8, device="cuda").t(), torch.uint8, 1, "x")
