"""The allocation-free Morton sort (dzs_morton_sort_noalloc) against the
oracle's Morton key and stable order (oracle.sort).

For callers that cannot allocate device memory (their device memory belongs to
a host framework's allocator, or they must not synchronise the device), the
library offers one sort whose scratch is a static device array.  This file is
collected last on purpose.  It must pass alone in a fresh process and after
every other test: two calls in a row, each compared bit for bit (index and
key work) with the oracle's permutation and keys of the same positions."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TWO32 = 2 ** 32


@pytest.fixture(scope="module")
def dzs():
    from paper_2005_05328_gb300 import build
    build.build()
    import paper_2005_05328_gb300 as m
    m.load()
    return m


def test_noalloc_sort_matches_the_oracle_twice(dzs):
    import torch

    import oracle as O
    dev = torch.device("cuda:0")
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(2024)
    sizes = [dzs.NOALLOC_SORT_MAX_N, 150001]
    perm_dev = torch.empty(dzs.NOALLOC_SORT_MAX_N, dtype=torch.int32, device=dev)
    keys_dev = torch.empty(dzs.NOALLOC_SORT_MAX_N, dtype=torch.int64, device=dev)
    for call, n in enumerate(sizes):
        u = rng.integers(0, TWO32, size=(3, n), dtype=np.uint64).astype(np.uint32)
        u[:, 100:400] = u[:, 1000:1300]  # equal keys: the order of ties is part of the result
        u_dev = torch.from_numpy(u.view(np.int32).copy()).to(dev)
        torch.cuda.synchronize()
        alloc_before = torch.cuda.memory_allocated(0), torch.cuda.memory_reserved(0)
        free_before = torch.cuda.mem_get_info(0)[0]
        status = dzs.dzs_morton_sort_noalloc(u_dev.data_ptr(), n, perm_dev.data_ptr(), keys_dev.data_ptr(),
                                             stream)
        assert status == dzs.DZS_OK
        torch.cuda.synchronize()
        # nothing allocated: torch's allocator untouched; device-wide free
        # memory (shared with the driver and other processes) within 2 MiB
        assert (torch.cuda.memory_allocated(0), torch.cuda.memory_reserved(0)) == alloc_before
        assert torch.cuda.mem_get_info(0)[0] >= free_before - (2 << 20)
        got = perm_dev[:n].cpu().numpy().view(np.uint32)
        key, perm = O.sort(u)
        assert np.array_equal(got, perm.astype(np.uint32)), call
        keys = keys_dev[:n].cpu().numpy().view(np.uint64)
        assert np.array_equal(keys, key[perm]), call


def test_noalloc_sort_rejects_oversize(dzs):
    import torch
    torch.cuda.set_device(0)
    n = dzs.NOALLOC_SORT_MAX_N + 1
    status = dzs.dzs_morton_sort_noalloc(1, n, 1, 0, 0)  # rejected before any pointer is used
    assert status == dzs.DZS_EINVAL
