"""Recoverable lightcone-ring overflow and host-side allocation-failure
injection (no GPU fault is involved in either).

Ring: a lightcone ring smaller than one step's crossings makes dzs_step stop
before the step that would not fit (DZS_EOVERFLOW, recoverable); after a
drain the next dzs_step resumes with that step.  The records, the final state
and the diagnostics are bit-identical to a run with the default ring (every
particle recorded once, none dropped; the particles cross the lightcone as the
paper's Sec. 1 footnote and Sec. 3.1.3 describe).

Allocation: the test hook makes the k-th device allocation fail; the failing
call returns DZS_ENOMEM, leaks nothing, and the library keeps working."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SMALL = dict(n1d=16, mesh=32, box=32.0, merge_level=2)


@pytest.fixture(scope="module")
def dzs():
    from paper_2005_05328_gb300 import build
    build.build()
    import paper_2005_05328_gb300 as m
    m.load()
    return m


@pytest.mark.parametrize("precision", [0, 1])
def test_small_ring_overflow_is_recoverable(dzs, precision):
    kw = dict(SMALL, precision=precision)
    with dzs.Context(**kw) as ctx:
        ctx.ics()
        assert ctx.step(96) == 96
        want = ctx.drain()
        want_state = ctx.state()
        want_diag = ctx.diagnostics()
        assert ctx.counters()[5] == 16 ** 3
    # the largest number of records one step writes, then a ring a little
    # larger than that (so every step fits after a drain) but far smaller
    # than the run's 4096 records
    per_step = []
    with dzs.Context(**kw) as ctx:
        ctx.ics()
        for _ in range(96):
            ctx.step(1)
            per_step.append(len(ctx.drain()))
    cap = max(per_step) + 8
    assert cap < 16 ** 3 // 4
    got, overflows, last_refused = [], 0, -1
    with dzs.Context(**dict(kw, lc_capacity=cap)) as ctx:
        ctx.ics()
        while ctx.count()[1] < 96:
            try:
                ctx.step(96)
            except dzs.DzsError as ex:
                assert ex.status == dzs.DZS_EOVERFLOW, ex
                overflows += 1
                step_before = ctx.count()[1]
                assert step_before != last_refused  # a drained ring always takes the next step
                last_refused = step_before
                got.append(ctx.drain(cap=cap))
                # the refused step had not started
                assert ctx.count()[1] == step_before
        got.append(ctx.drain(cap=cap))
        state = ctx.state()
        diag = ctx.diagnostics()
        cnt = ctx.counters()
    assert overflows > 0
    rec = np.concatenate(got)
    assert rec.tobytes() == want.tobytes()
    for key in want_state:
        assert np.array_equal(state[key], want_state[key]), key
    assert np.array_equal(diag, want_diag)
    assert cnt[3] & 4 == 0  # no ring-full error bit: no record dropped


def test_allocation_failure_is_reported_and_leaks_nothing(dzs):
    import torch
    torch.cuda.set_device(0)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(0)[0]
    dzs.dzs_debug_fail_alloc(1)  # the context's arena
    with pytest.raises(dzs.DzsError) as ex:
        dzs.Context(**SMALL)
    assert ex.value.status == dzs.DZS_ENOMEM
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(0)[0] >= free0 - (2 << 20)
    # the hook is spent: the next context works, and an observer whose second
    # buffer fails frees the first
    with dzs.Context(**SMALL) as ctx:
        ctx.ics()
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info(0)[0]
        dzs.dzs_debug_fail_alloc(2)
        with pytest.raises(dzs.DzsError) as ex:
            ctx.observe(nside=64, mesh=64)
        assert ex.value.status == dzs.DZS_ENOMEM
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info(0)[0] >= free1 - (2 << 20)
        dzs.dzs_debug_fail_alloc(0)
        ctx.observe(nside=64, mesh=64)
        ctx.step(2)
        assert ctx.count()[1] == 2
