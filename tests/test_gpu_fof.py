"""GPU parity of the friends-of-friends haloes (Sec. 3.1.1) against the oracle:
membership (labels), counts, masses and observer distances bit-exact (integer
work); centres of mass bit-exact (the same exact integer sums and the same
correctly rounded FP64 operations).  The caller's particle order is kept."""
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


def compare(h, lab, wh, wlab):
    assert np.array_equal(lab, wlab)
    assert len(h) == len(wh) > 0
    for f in ("first", "count", "mass", "rmax2"):
        assert np.array_equal(h[f], wh[f]), f
    assert np.array_equal(h["x"], wh["x"])


@pytest.mark.parametrize("upto,link,nmin", [(60, 0.35, 5), (75, 0.2, 2), (75, 0.35, 5), (90, 0.35, 2)])
def test_fof_matches_oracle(dzs, upto, link, nmin):
    P = O.params(**SMALL)
    st = O.initial_state(P)
    for n in range(upto):
        st, _ = O.step(P, n, st)
    perm = np.random.default_rng(upto).permutation(st["u"].shape[1])  # any caller order
    st = {f: (v[:, perm] if v.ndim == 2 else v[perm]) for f, v in st.items()}
    wh, wlab = O.fof(P, st["u"], st["k"], link=link, nmin=nmin)
    with dzs.Context(**SMALL, precision=0) as ctx:
        ctx.set_state(st, upto)
        before = ctx.state()
        h, lab = ctx.fof(link=link, nmin=nmin, labels=True)
        after = ctx.state()
    for f in before:
        assert np.array_equal(before[f], after[f]), f
    compare(h, lab, wh, wlab)


def test_fof_full_size_clustered(dzs):
    """2M particles in 256 Mpc/h (the bench workload's size), a third of them
    in Gaussian clumps of every size, multiplicities 1-8"""
    rng = np.random.default_rng(17)
    kw = dict(n1d=128, mesh=256, box=256.0, merge_level=3)
    P = O.params(**kw)
    n = 128 ** 3
    x = rng.uniform(0, 256.0, size=(3, n))
    m = n // 3
    nc = 3000
    sizes = rng.multinomial(m, rng.dirichlet(np.ones(nc) * 0.3))
    pos = 0
    for c in range(nc):
        s = sizes[c]
        x[:, pos:pos + s] = rng.uniform(0, 256.0, size=(3, 1)) + rng.normal(0, rng.uniform(0.1, 1.5),
                                                                              size=(3, s))
        pos += s
    u = (np.mod(x, 256.0) / 256.0 * TWO32).astype(np.uint64).astype(np.uint32)
    k = rng.integers(1, 9, size=n).astype(np.uint32)
    st = dict(u=u, p=np.zeros((3, n)), g=np.zeros((3, n)), k=k, id=np.arange(n, dtype=np.uint32),
              fl=np.zeros(n, np.uint8))
    wh, wlab = O.fof(P, u, k, link=0.2, nmin=20)
    with dzs.Context(**kw, precision=0) as ctx:
        ctx.set_state(st, 0)
        h, lab = ctx.fof(link=0.2, nmin=20, labels=True)
    compare(h, lab, wh, wlab)
    assert len(h) > 500


def test_fof_errors(dzs):
    with dzs.Context(**SMALL) as ctx:
        with pytest.raises(dzs.DzsError):
            ctx.fof()  # no state
        ctx.ics()
        for bad in (dict(link=0.0), dict(nmin=1), dict(link=20.0)):
            with pytest.raises(dzs.DzsError) as e:
                ctx.fof(**bad)
            assert e.value.status == dzs.DZS_EINVAL
