"""fmm_copy: SM-driven copies between device and pinned host memory (GPU)."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2302_07567_gb300 import fmm

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.int32])
def test_copies_equal_torch_copies(dtype):
    g = torch.Generator().manual_seed(5)
    host = (torch.randn((65536, 3), generator=g) * 1e3).to(dtype).pin_memory()
    d = torch.empty(host.shape, dtype=dtype, device=DEV)
    fmm.copy_(d, host)  # host -> device
    torch.cuda.synchronize()
    assert torch.equal(d.cpu(), host)
    d2 = torch.empty_like(d)
    fmm.copy_(d2, d)  # device -> device
    back = torch.empty(host.shape, dtype=dtype).pin_memory()
    fmm.copy_(back, d2)  # device -> host
    torch.cuda.synchronize()
    assert torch.equal(back, host)


def test_rejects_what_a_kernel_cannot_address():
    d = torch.empty((1024,), dtype=torch.float64, device=DEV)
    with pytest.raises(ValueError):
        fmm.copy_(d, torch.zeros(1024, dtype=torch.float64))  # pageable host memory
    with pytest.raises(ValueError):
        fmm.copy_(d, torch.zeros(1000, dtype=torch.float64).pin_memory())  # size differs
    # the library's own checks: pageable memory, a misaligned address
    page = np.zeros(1024)
    lib = fmm.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream)
    assert lib.fmm_copy(ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(page.ctypes.data), 8192, stream) == fmm.FMM_EINVAL
    assert lib.fmm_copy(ctypes.c_void_p(d.data_ptr() + 8), ctypes.c_void_p(d.data_ptr()), 4096, stream) == fmm.FMM_EINVAL
    torch.cuda.synchronize()
