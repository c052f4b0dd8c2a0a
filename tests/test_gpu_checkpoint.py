"""Checkpoint / restore (the adapted halt-and-restart of the paper, Sec. 4.1.1):
a run resumed from a checkpoint continues bit for bit, lightcone records
included, in a fresh context and in the same one (rewind)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KW = dict(n1d=16, mesh=32, box=32.0, merge_level=2, seed=7)


@pytest.fixture(scope="module")
def dzs():
    from paper_2005_05328_gb300 import build
    build.build()
    import paper_2005_05328_gb300 as m
    m.load()
    return m


def run_and_collect(ctx, steps):
    ctx.step(steps)
    return ctx.state(), ctx.drain()


@pytest.mark.parametrize("precision", [0, 1])
def test_resume_is_bit_identical(dzs, precision):
    with dzs.Context(**KW, precision=precision) as a:
        a.ics()
        a.step(50)
        part = a.drain(cap=1 << 16)  # drain some records before the checkpoint
        a.step(5)                    # leave records pending in the ring
        blob = a.checkpoint()
        st_a, rec_a = run_and_collect(a, 20)
        # rewind the same context
        a.restore(blob)
        st_r, rec_r = run_and_collect(a, 20)
    with dzs.Context(**KW, precision=precision) as b:
        b.restore(blob)
        assert b.count()[1] == 55
        st_b, rec_b = run_and_collect(b, 20)
    assert len(part) > 0
    for st, rec in ((st_r, rec_r), (st_b, rec_b)):
        for name in st_a:
            assert np.array_equal(st[name], st_a[name]), name
        assert rec.tobytes() == rec_a.tobytes()


def test_restore_rejects_mismatch(dzs):
    with dzs.Context(**KW) as a:
        a.ics()
        blob = a.checkpoint()
    with dzs.Context(**dict(KW, merge_level=1)) as b:
        with pytest.raises(dzs.DzsError) as e:
            b.restore(blob)
        assert e.value.status == dzs.DZS_EINVAL
    with dzs.Context(**KW) as c:
        with pytest.raises(dzs.DzsError):
            c.restore(blob[:100])
        bad = bytearray(blob)
        bad[0] ^= 0xFF
        with pytest.raises(dzs.DzsError):
            c.restore(bytes(bad))
