"""The device oct-tree against its definition (Sec. 2.1: the root is the box;
a node holding more than B particles splits into its non-empty octants, down
to depth 21; the walk groups are the nodes with <= G particles whose parent
holds more, or leaves whose parent holds more).

The node count and the group count of the CUDA tree (built without a pass per
depth) equal those of a plain recursive top-down split of the sorted keys
written here, and the group count equals the oracle's; inputs: clustered sets
of several sizes, B and G, sets of at most B and at most G particles, runs of
coincident particles, and a lattice.  The number of (particle, list entry)
pairs the walk evaluates equals the oracle's interaction count exactly (the
same interaction sets, whatever node the walk starts from), and the
accelerations through the same tree match the oracle (FP64) on each input."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

TWO32 = 2 ** 32
SMALL = dict(n1d=32, mesh=64, box=64.0, merge_level=2)  # capacity 32^3 >= every case


@pytest.fixture(scope="module")
def dzs():
    from paper_2005_05328_gb300 import build
    build.build()
    import paper_2005_05328_gb300 as m
    m.load()
    return m


def morton_sorted(u):
    keys = np.array([O.morton_key(*u[:, i]) for i in range(u.shape[1])], dtype=np.uint64)
    order = np.argsort(keys, kind="stable")
    return u[:, order], keys[order]


def top_down(keys, B, G):
    """(nodes, groups) of the recursive split: a node [s, e) at depth j splits
    when e - s > B and j < 21 into the runs of equal digit j + 1"""
    nodes = groups = 0
    n = len(keys)
    if n == 0:
        return 0, 0
    stack = [(0, n, 0, True)]  # start, end, depth, parent holds more than G
    while stack:
        s, e, j, big_parent = stack.pop()
        nodes += 1
        leaf = e - s <= B or j == 21
        if big_parent and (e - s <= G or leaf):
            groups += 1
        if leaf:
            continue
        d = (keys[s:e] >> np.uint64(3 * (20 - j))) & np.uint64(7)
        cuts = np.flatnonzero(np.diff(d)) + 1
        bounds = [s] + list(s + cuts) + [e]
        for a, b in zip(bounds[:-1], bounds[1:]):
            stack.append((a, b, j + 1, e - s > G))
    return nodes, groups


def clustered(rng, n, nclump, spread):
    x = rng.uniform(0, 1, size=(3, n))
    m = n // 2
    for c in range(nclump):
        sl = slice(c * m // nclump, (c + 1) * m // nclump)
        x[:, sl] = rng.uniform(0, 1, size=(3, 1)) + rng.normal(0, spread, size=(3, sl.stop - sl.start))
    return (np.mod(x, 1.0) * TWO32).astype(np.uint64).astype(np.uint32)


def cases():
    rng = np.random.default_rng(41)
    out = [("clustered 3000", clustered(rng, 3000, 5, 0.01), {}),
           ("clustered 20000", clustered(rng, 20000, 12, 0.003), {}),
           ("clustered B=4 G=16", clustered(rng, 5000, 6, 0.005), dict(leaf_bucket=4, walk_group=16)),
           ("clustered B=14 G=64", clustered(rng, 5000, 6, 0.005), dict(leaf_bucket=14, walk_group=64)),
           ("n = B", clustered(rng, 8, 1, 0.01), {}),
           ("n = G", clustered(rng, 32, 1, 0.01), {}),
           ("n = G + 1", clustered(rng, 33, 1, 0.001), {})]
    # runs of coincident particles (equal keys) among scattered ones
    u = clustered(rng, 2000, 4, 0.01)
    u[:, 100:140] = u[:, 100:101]
    u[:, 500:509] = u[:, 500:501]
    out.append(("coincident runs", u, {}))
    # a 16^3 lattice: every depth-4 cell holds 8 particles
    g = (np.arange(16, dtype=np.uint64) * (TWO32 // 16) + 12345)
    out.append(("lattice", np.array(np.meshgrid(g, g, g, indexing="ij")).reshape(3, -1).astype(np.uint32), {}))
    return out


@pytest.mark.parametrize("name,u,extra", cases(), ids=[c[0] for c in cases()])
def test_tree_counts_match_definition(dzs, name, u, extra):
    kw = dict(SMALL, **extra)
    P = O.params(**kw)
    us, keys = morton_sorted(u)
    nodes, groups = top_down(keys, P.leaf_bucket, P.walk_group)
    st, ct = O.groups(P, us)
    assert len(st) == groups and ct.sum() == us.shape[1]
    n = us.shape[1]
    state = dict(u=us, p=np.zeros((3, n)), g=np.zeros((3, n)), k=np.ones(n, np.uint32),
                 id=np.arange(n, dtype=np.uint32), fl=np.zeros(n, np.uint8))
    want = O.accel(P, us, state["k"])
    with dzs.Context(**kw, precision=1) as ctx:
        ctx.set_state(state, 0)
        got = ctx.accel()
        cnt = ctx.counters()
    assert cnt[3] == 0
    assert cnt[0] == groups, (name, cnt[0], groups)
    assert cnt[1] == nodes, (name, cnt[1], nodes)
    # the interaction set: every particle's list length summed, exactly the
    # oracle's (monopoles and leaf particles per group, times its particles)
    assert cnt[2] == O.interaction_count(P, us, state["k"]), (name, cnt[2])
    # a lattice's exact force is 0: scale by the pair force at the mean spacing,
    # G m0 / (L / N1)^2, G m0 = 1.5 Omega_m L^3 / (4 pi N1^3)
    spacing = kw["box"] / kw["n1d"]
    scale = max(np.abs(want).max(), 1.5 * P.omega_m * kw["box"] ** 3 / (4 * np.pi * kw["n1d"] ** 3) / spacing ** 2)
    assert np.abs(got - want).max() <= 1e-9 * scale
