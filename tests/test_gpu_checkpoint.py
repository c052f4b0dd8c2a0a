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


KW2 = dict(n1d=32, mesh=64, box=64.0, merge_level=3, seed=7)


@pytest.mark.parametrize("precision", [0, 1])
def test_halt_shrink_resume_is_bit_identical(dzs, precision):
    """Sec. 4.1.1 adapted: halt once N / N0 < 0.5, checkpoint, re-create the
    context with only the slots the particles need, restore, finish the run;
    state and lightcone equal those of an uninterrupted run bit for bit."""
    with dzs.Context(**KW2, precision=precision) as ref:
        ref.ics()
        ref.step(96)
        st_ref, rec_ref = ref.state(), ref.drain()
    with dzs.Context(**KW2, precision=precision) as a:
        a.ics()
        done, why, r = a.step_until(96, ratio_min=0.5)
        assert why == dzs.HALT_RATIO and r < 0.5 and 0 < done < 96
        n, step = a.count()
        assert step == done and n / 32 ** 3 == r
        rec1 = a.drain()
        blob = a.checkpoint()
    full = dzs.dzs_footprint_bytes(dzs.params(**KW2, precision=precision))
    shrunk = dzs.dzs_footprint_bytes(dzs.params(**KW2, precision=precision, capacity=n))
    assert shrunk < full
    with dzs.Context(**KW2, precision=precision, capacity=n) as b:
        with pytest.raises(dzs.DzsError):
            b.ics()  # the ICs need all n1d^3 slots
        b.restore(blob)
        b.step(96)
        st_b, rec2 = b.state(), b.drain()
    for name in st_ref:
        assert np.array_equal(st_b[name], st_ref[name]), name
    assert np.concatenate([rec1, rec2]).tobytes() == rec_ref.tobytes()


def test_wall_limit_halts(dzs):
    with dzs.Context(**KW2) as a:
        a.ics()
        done, why, r = a.step_until(96, ratio_min=0.5, wall_limit_s=1e-9, horizon_s=1e9)
        assert done == 1 and why == dzs.HALT_WALL and r == 1.0  # R flat: no re-allocation due
        done, why, r = a.step_until(96, ratio_min=0.9)
        assert why == dzs.HALT_RATIO
        # while R falls, the extrapolation at the limit crosses 0.5 within the horizon
        fell = False
        for _ in range(10):
            done, why, r2 = a.step_until(96, ratio_min=0.5, wall_limit_s=1e-9, horizon_s=1e9)
            assert done == 1
            if r2 < r:
                fell = True
                assert why == dzs.HALT_PREDICTED or (why == dzs.HALT_RATIO and r2 < 0.5)
            else:
                assert why == dzs.HALT_WALL
            r = r2
        assert fell
