"""The walk's two frontiers build the interaction sets of a walk from the root
(Sec. 2.1, Eq. 1 per walk group, the r_cut skip).

A group walk may start from the depth-F nodes of the cells within r_cut of
the group cube along each axis instead of the 27 depth-f cells around it,
when every ancestor of those nodes between depths f and F opens for any group
cube that does not skip it.  Then the walk from f would open or skip each of
those ancestors, and exactly the same nodes get tested: the number of
(particle, list entry) pairs equals the oracle's interaction count (a walk
from the root, one recursion per group) exactly, and the accelerations match
the oracle (FP64 1e-9 of the largest, FP32 99.9th percentile 1e-4).  Inputs:
Zel'dovich sets at z = 49 (near a lattice: every group takes the window) and
at z = 0.3 (shell-crossed, clustered: some groups fall back), a set with
random multiplicities k in 1..8 (COMs off the cell centres), and one with the
bench mock's geometry (spacing 2 Mpc/h, r_cut = 5.625 Mpc/h)."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dzs():
    from paper_2005_05328_gb300 import build
    build.build()
    import paper_2005_05328_gb300 as m
    m.load()
    return m


CASES = {
    "32cubed_z49": (dict(n1d=32, mesh=64, box=64.0), 49.0, False),
    "32cubed_z0.3": (dict(n1d=32, mesh=64, box=64.0), 0.3, False),
    "32cubed_z0.3_k1to8": (dict(n1d=32, mesh=64, box=64.0), 0.3, True),
    "64cubed_z2": (dict(n1d=64, mesh=128, box=128.0), 2.0, False),
}


def sorted_state(kw, z, multi):
    P = O.params(**kw, z_init=z)
    s = O.ics(P)
    _, perm = O.sort(s["u"])
    u = np.ascontiguousarray(s["u"][:, perm])
    n = u.shape[1]
    k = np.ones(n, np.uint32)
    if multi:
        k = np.random.default_rng(7).integers(1, 9, size=n).astype(np.uint32)
    st = dict(u=u, p=np.zeros((3, n)), g=np.zeros((3, n)), k=k, id=np.arange(n, dtype=np.uint32),
              fl=np.zeros(n, np.uint8))
    return P, st


@pytest.mark.parametrize("name", list(CASES))
def test_window_frontier_builds_the_root_walk_sets(dzs, name):
    kw, z, multi = CASES[name]
    P, st = sorted_state(kw, z, multi)
    n = st["u"].shape[1]
    sample = None if n <= 32 ** 3 else np.random.default_rng(3).choice(n, 3000, replace=False)
    want = O.accel(P, st["u"], st["k"], sample=sample)
    idx = np.arange(n) if sample is None else sample
    for precision in (1, 0):
        with dzs.Context(**kw, z_init=z, precision=precision) as ctx:
            ctx.set_state(st, 0)
            got = ctx.accel()
            cnt = ctx.counters()
            wc = ctx.walk_counters()
        assert cnt[3] == 0
        assert wc[4] > 0, wc  # the window frontier was taken
        assert cnt[2] == O.interaction_count(P, st["u"], st["k"]), (name, precision, cnt[2])
        e = np.linalg.norm(got[:, idx] - want[:, idx], axis=0)
        ref = np.linalg.norm(want[:, idx], axis=0)
        rel = e / (ref + 1e-3 * np.sqrt((ref ** 2).mean()))
        if precision == 1:
            assert e.max() <= 1e-9 * ref.max(), (name, e.max() / ref.max())
        else:
            assert np.percentile(rel, 99.9) <= 1e-4, (name, np.percentile(rel, 99.9))
        print(name, "precision", precision, "window", int(wc[4]), "fallback", int(wc[5]))


def test_walk_diagnostics_are_opt_in(dzs):
    """node tests, rounds and stack depth are counted only with the walk
    diagnostics flag; the accelerations do not depend on it"""
    kw, z, multi = CASES["32cubed_z0.3"]
    P, st = sorted_state(kw, z, multi)
    out = {}
    for diag in (False, True):
        with dzs.Context(**kw, z_init=z, precision=0) as ctx:
            ctx.set_state(st, 0)
            ctx.set_profiling(True, walk_diag=diag)
            g = ctx.accel()
            out[diag] = (g, ctx.walk_counters(), ctx.counters())
    assert np.array_equal(out[False][0], out[True][0])
    assert out[False][1][2] == 0 and out[False][1][3] == 0 and out[False][2][6] == 0
    assert out[True][1][2] > 0 and out[True][1][3] > 0 and out[True][2][6] > 0
    assert np.array_equal(out[False][1][[0, 1, 4, 5]], out[True][1][[0, 1, 4, 5]])
