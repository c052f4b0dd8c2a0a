"""Degenerate inputs through the CUDA path: an empty particle set, a single
particle, coincident particles (one depth-21 leaf with more than B members),
particles at the lattice corners (periodic wrap), and the end of the run.
Each must run, conserve what it should and agree with the oracle where the
oracle defines the answer."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

TWO32 = 2 ** 32
SMALL = dict(n1d=16, mesh=32, box=32.0, merge_level=2)


@pytest.fixture(scope="module")
def dzs():
    from paper_2005_05328_gb300 import build
    build.build()
    import paper_2005_05328_gb300 as m
    m.load()
    return m


def state(u, k=None, p=None):
    n = u.shape[1]
    return dict(u=u.astype(np.uint32), p=np.zeros((3, n)) if p is None else p, g=np.zeros((3, n)),
                k=np.ones(n, np.uint32) if k is None else k, id=np.arange(n, dtype=np.uint32),
                fl=np.zeros(n, np.uint8))


@pytest.mark.parametrize("precision", [0, 1])
def test_empty_set(dzs, precision):
    with dzs.Context(**SMALL, precision=precision) as ctx:
        ctx.set_state(state(np.zeros((3, 0), np.uint32)), 10)
        ctx.step(3)
        n, step = ctx.count()
        assert n == 0 and step == 13
        assert len(ctx.drain()) == 0
        d = ctx.diagnostics()
        assert d[0] == 0 and d[7] == 0
        k, p, m = ctx.power_spectrum(4)
        assert np.all(m > 0)
        assert len(ctx.fof(nmin=2)) == 0


@pytest.mark.parametrize("precision", [0, 1])
def test_single_particle(dzs, precision):
    P = O.params(**SMALL)
    u = np.array([[123456789], [987654321], [2 ** 31 + 5]], np.uint64)
    st = state(u, k=np.array([7], np.uint32), p=np.array([[0.1], [-0.2], [0.3]]))
    want = O.accel(P, st["u"], st["k"])
    with dzs.Context(**SMALL, precision=precision) as ctx:
        ctx.set_state(st, 0)
        g = ctx.accel()
        # the exact answer is 0 (no other mass, no self force): compare with the
        # particle's own force scale at one mesh spacing, G m k / Delta^2
        scale = 1.5 * P.omega_m * P.box ** 3 / (4 * np.pi * 16 ** 3) * 7 / (P.box / P.mesh) ** 2
        assert np.abs(g - want).max() <= (1e-12 if precision == 1 else 1e-6) * scale
        ctx.step(2)
        d = ctx.diagnostics()
        assert d[0] == 7 and d[7] == 1


def test_coincident_particles_one_leaf(dzs):
    """64 particles on one lattice point: one depth-21 leaf with more than B
    members (streamed through the walk), zero pair forces among them"""
    P = O.params(**SMALL)
    u = np.full((3, 64), 2 ** 30, np.uint64)
    u = np.concatenate([u, np.array([[2 ** 30 + 2 ** 24], [2 ** 30], [2 ** 30]], np.uint64)], axis=1)
    st = state(u)
    want = O.accel(P, st["u"], st["k"], parts=2)
    with dzs.Context(**SMALL, precision=1) as ctx:
        ctx.set_state(st, 0)
        got = ctx.accel(dzs.ACC_TREE)
        cnt = ctx.counters()
    assert np.allclose(got, want, rtol=1e-9, atol=1e-12 * np.abs(want).max())
    assert cnt[3] == 0


def test_corner_particles_wrap(dzs):
    """particles at the eight lattice corners are one periodic clump"""
    P = O.params(**SMALL)
    c = [0, TWO32 - 1]
    pts = [(x, y, z) for x in c for y in c for z in c]
    u = np.array(pts, np.uint64).T
    st = state(u)
    want = O.accel(P, st["u"], st["k"])
    with dzs.Context(**SMALL, precision=1) as ctx:
        ctx.set_state(st, 0)
        got = ctx.accel()
        h = ctx.fof(link=0.01, nmin=8)
    err = np.linalg.norm(got - want, axis=0) / (np.linalg.norm(want, axis=0) + 1e-3 * np.abs(want).max())
    assert err.max() <= 1e-9
    assert len(h) == 1 and h["count"][0] == 8


def test_run_ends_at_a_equals_one(dzs):
    with dzs.Context(**SMALL) as ctx:
        ctx.ics()
        assert ctx.step(1000) == 96
        assert ctx.step(1) == 0
        with pytest.raises(dzs.DzsError) as e:
            ctx.run_stages(dzs.STAGE_ALL)
        assert e.value.status == dzs.DZS_ESTATE
