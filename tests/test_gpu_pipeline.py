"""Pipelined per-step results (dzs_pipeline / dzs_step_result /
dzs_lightcone_drain_step): reading step s while step s + 1 runs returns
exactly what the synchronous calls return after each step — the conservation
diagnostics of Sec. 2.1/2.2 (Sigma k, Sigma k p, Sigma k u, N) bit for bit,
and the same lightcone records in the same order — and the state after the
run is bit-identical.  Only the last 4 steps are kept; asking for another is
an error, as is asking with pipelining off."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KW = dict(n1d=32, mesh=64, box=64.0, merge_level=2, seed=5)


@pytest.fixture(scope="module")
def dzs():
    from paper_2005_05328_gb300 import build
    build.build()
    import paper_2005_05328_gb300 as m
    m.load()
    return m


def test_pipelined_results_match_the_synchronous_ones(dzs):
    steps = 40
    sync_diag, sync_rec = [], []
    with dzs.Context(**KW) as ctx:
        ctx.ics()
        for _ in range(steps):
            ctx.step(1)
            sync_rec.append(ctx.drain(cap=32 ** 3))
            sync_diag.append(ctx.diagnostics())
        sync_state = ctx.state()
    pipe_diag, pipe_rec = [], []
    with dzs.Context(**KW) as ctx:
        ctx.ics()
        ctx.pipeline(True)
        ctx.step(1)
        for s in range(1, steps + 1):
            if s < steps:
                ctx.step(1)  # step s + 1 is queued before step s is read
            pipe_rec.append(ctx.drain_step(s, cap=32 ** 3))
            d, written = ctx.step_result(s)
            pipe_diag.append(d)
            assert written == sum(len(r) for r in pipe_rec)
        ctx.pipeline(False)
        pipe_state = ctx.state()
    for s in range(steps):
        assert np.array_equal(pipe_diag[s], sync_diag[s]), s
        assert np.array_equal(pipe_rec[s], sync_rec[s]), s
    assert sum(len(r) for r in pipe_rec) > 0
    for name in ("u", "p", "k", "id", "fl"):
        assert np.array_equal(pipe_state[name], sync_state[name]), name


def test_pipelined_result_bookkeeping(dzs):
    with dzs.Context(**KW) as ctx:
        ctx.ics()
        with pytest.raises(dzs.DzsError):
            ctx.step_result(0)  # pipelining off
        ctx.pipeline(True)
        ctx.step(6)
        for s in (3, 4, 5, 6):
            d, _ = ctx.step_result(s)
            assert d[0] == 32 ** 3  # mass is conserved exactly
        for s in (1, 2, 7):
            with pytest.raises(dzs.DzsError):
                ctx.step_result(s)  # not kept, or not run
        ctx.pipeline(False)
