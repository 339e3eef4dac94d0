"""The device generators fill HBM with the same fp32 values as the host ones (the
seeded inputs every parity test and the benchmark share)."""
import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    return torch


@pytest.mark.parametrize("length", [256, 100, 1024])
def test_device_walks_and_mixed_equal_host(torch_cuda, length):
    torch = torch_cuda
    count, first = 777, 12345
    for fn_dev, fn_host, seed in ((datagen.walks_device, datagen.walks, 3), (datagen.mixed_device, datagen.mixed, 4)):
        out = torch.empty((count, length), dtype=torch.float32, device="cuda")
        fn_dev(seed, first, count, length, out.data_ptr(), 0)
        torch.cuda.synchronize()
        host = fn_host(seed, first, count, length)
        assert np.array_equal(out.cpu().numpy().view(np.uint32), host.view(np.uint32)), fn_host.__name__
