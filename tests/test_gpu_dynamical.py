"""GPU parity of the dynamical DZS criterion (Sec. 2.2.1: Eq. 2 with the node
distance of Eq. 3, a_min over the particles not yet crossed) against the FP64
oracle.  Merge membership, masses, COM positions, ids and flags are
bit-exact: the kernel takes every FP64 operation of the decision with a
correctly rounded intrinsic in the oracle's order, and a_min^2 from the same
accelerations (rounded to FP32 first for an FP32 context)."""
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


def oparams(**kw):
    kw = dict(kw)
    kw.pop("precision", None)
    if "dzs_criterion" in kw:
        kw["criterion"] = kw.pop("dzs_criterion")
    return O.params(**kw)


_cache = {}


def evolved(upto):
    """un-merged oracle state after `upto` steps (cached)"""
    if upto not in _cache:
        P = oparams(**SMALL, dzs_on=0)
        st = O.initial_state(P)
        for n in range(upto):
            st, _ = O.step(P, n, st)
        _cache[upto] = st
    return _cache[upto]


def d2_obs(u):
    off = u.astype(np.int64) - 2 ** 31
    return (off ** 2).sum(axis=0).astype(np.uint64)


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("upto,rfrac", [(70, 0.1), (80, 0.2), (90, 0.15)])
def test_dynamical_merge_bit_exact(dzs, precision, upto, rfrac):
    st = dict(evolved(upto))
    rlat = int(rfrac * TWO32)
    # particles beyond R have crossed; a_min comes from the ones inside
    fl = np.where(d2_obs(st["u"]) >= np.uint64(rlat) ** 2, O.FL_CROSSED, 0).astype(np.uint8)
    st["fl"] = fl
    assert 0 < (fl == 0).sum() < len(fl)
    if precision == 0:
        st["p"] = st["p"].astype(np.float32).astype(np.float64)
        st["g"] = st["g"].astype(np.float32).astype(np.float64)
    counts = []
    for alpha in (1e-3, 1e-1, 10.0, 1e3):
        kw = dict(SMALL, dzs_criterion=1, alpha_dyn=alpha)
        want = O.merge(oparams(**kw), rlat, st)
        with dzs.Context(**dict(kw, precision=precision)) as ctx:
            ctx.set_state(st, upto)
            ctx.merge_only(rlat)
            got = ctx.state()
        for name in ("u", "k", "id", "fl"):
            assert np.array_equal(got[name], want[name]), (alpha, name)
        if precision == 1:
            assert np.array_equal(got["p"], want["p"])
        else:
            assert np.array_equal(got["p"], want["p"].astype(np.float32).astype(np.float64))
        counts.append(want["u"].shape[1])
    n = st["u"].shape[1]
    assert all(b <= a for a, b in zip(counts, counts[1:]))
    assert counts[-1] < counts[0] and counts[-1] < n


def test_dynamical_no_uncrossed_is_infinite_amin(dzs):
    """every particle crossed: a_min = infinity, so every cell with D > 0
    merges (alpha > 0) and none does at alpha = 0"""
    st = dict(evolved(70))
    st["fl"] = np.full_like(st["fl"], O.FL_CROSSED)
    rlat = int(0.1 * TWO32)
    for alpha in (0.0, 0.5):
        kw = dict(SMALL, dzs_criterion=1, alpha_dyn=alpha)
        want = O.merge(oparams(**kw), rlat, st)
        with dzs.Context(**dict(kw, precision=1)) as ctx:
            ctx.set_state(st, 70)
            ctx.merge_only(rlat)
            got = ctx.state()
        for name in ("u", "p", "k", "id", "fl"):
            assert np.array_equal(got[name], want[name]), (alpha, name)
        if alpha == 0.0:
            assert got["u"].shape[1] == st["u"].shape[1]
        else:
            assert got["u"].shape[1] < st["u"].shape[1]


@pytest.mark.parametrize("upto", [60, 85])
def test_dynamical_full_step_fp64(dzs, upto):
    kw = dict(SMALL, dzs_criterion=1, alpha_dyn=0.05)
    P = oparams(**kw)
    st = evolved(upto)
    so, rec = O.step(P, upto, st)
    with dzs.Context(**dict(kw, precision=1)) as ctx:
        ctx.set_state(st, upto)
        ctx.step(1)
        s = ctx.state()
        r = ctx.drain()
    assert np.array_equal(np.sort(r["id"]), np.sort(rec["id"]))
    assert np.array_equal(s["id"], so["id"]) and np.array_equal(s["k"], so["k"])
    assert np.array_equal(s["fl"], so["fl"])
    du = (s["u"].astype(np.int64) - so["u"].astype(np.int64) + 2 ** 31) % TWO32 - 2 ** 31
    assert np.abs(du).max() <= 1
