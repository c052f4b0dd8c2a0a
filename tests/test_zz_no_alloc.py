"""The allocation-free Morton sort (dzs_morton_sort_noalloc) against the
step's own sort entry point (dzs_run_stages with DZS_STAGE_SORT).

For callers that cannot allocate device memory (their device memory belongs to
a host framework's allocator, or they must not synchronise the device), the
library offers one sort whose scratch is a static device array.  This file is
collected last on purpose.  It must pass alone in a fresh process and after
every other test: two calls in a row, each compared bit for bit (index work)
with the context-based sort of the same positions."""
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


def reference_perm(dzs, u):
    """Permutation from the existing context sort: inject ids 0..n-1, sort,
    read the ids back in sorted order."""
    n = u.shape[1]
    st = dict(u=u, p=np.zeros((3, n)), g=np.zeros((3, n)), k=np.ones(n, np.uint32),
              id=np.arange(n, dtype=np.uint32), fl=np.zeros(n, np.uint8))
    with dzs.Context(n1d=64, mesh=64, box=128.0) as ctx:  # N0 = 262144 >= n
        ctx.set_state(st, 0)
        ctx.run_stages(dzs.STAGE_SORT)
        return ctx.state()["id"]


def test_noalloc_sort_matches_context_sort_twice(dzs):
    import torch
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
        if call == 1:
            free_before = torch.cuda.mem_get_info(0)[0]
        status = dzs.dzs_morton_sort_noalloc(u_dev.data_ptr(), n, perm_dev.data_ptr(), keys_dev.data_ptr(),
                                             stream)
        assert status == dzs.DZS_OK
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info(0)[0] == free_before  # nothing allocated
        got = perm_dev[:n].cpu().numpy().view(np.uint32)
        want = reference_perm(dzs, u)
        assert np.array_equal(got, want), call
        keys = keys_dev[:n].cpu().numpy().view(np.uint64)
        assert np.all(keys[1:] >= keys[:-1])


def test_noalloc_sort_rejects_oversize(dzs):
    import torch
    torch.cuda.set_device(0)
    n = dzs.NOALLOC_SORT_MAX_N + 1
    status = dzs.dzs_morton_sort_noalloc(1, n, 1, 0, 0)  # rejected before any pointer is used
    assert status == dzs.DZS_EINVAL
