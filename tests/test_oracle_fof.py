"""Pins of the oracle's friends-of-friends haloes (oracle/fof.c; paper Sec.
3.1.1, the lightcone halo mass function from FoF catalogues).

Pins: the components equal those of the exact integer friends graph computed
by brute force and scipy's connected_components (both the all-pairs and the
grid paths of the oracle); the linking threshold is inclusive at exactly the
linking length and exclusive one lattice unit beyond; a clump straddling the
periodic boundary is one halo with its centre of mass on the right side; a
symmetric clump has its centre of mass at its centre; masses, counts and the
largest distance from the observer follow their definitions; nmin filters."""
import math

import numpy as np
import pytest

import oracle as O

TWO32 = 2 ** 32


def brute_components(u, T):
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    n = u.shape[1]
    ui = u.astype(np.int64)
    rows, cols = [], []
    for i in range(n):
        d = ((ui[:, i + 1:] - ui[:, i:i + 1] + 2 ** 31) % TWO32) - 2 ** 31
        d2 = (d.astype(np.int64) ** 2).astype(np.uint64).sum(axis=0)  # exact: < 3 2^62
        js = np.nonzero(d2 <= np.uint64(T))[0] + i + 1
        rows += [i] * len(js)
        cols += js.tolist()
    g = coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    _, lab = connected_components(g, directed=False)
    # relabel each component by its smallest member
    first = {}
    for i in range(n):
        first.setdefault(lab[i], i)
    return np.array([first[x] for x in lab])


@pytest.mark.parametrize("n,link,nside", [(250, 0.9, 8), (3000, 0.5, 16), (6000, 0.4, 16)])
def test_components_match_brute_force(n, link, nside):
    rng = np.random.default_rng(n)
    P = O.params(n1d=nside, mesh=2 * nside, box=2.0 * nside)
    # clumpy: half the points in a few Gaussian blobs
    x = rng.uniform(0, P.box, size=(3, n))
    m = n // 2
    for c in range(5):
        sl = slice(c * m // 5, (c + 1) * m // 5)
        x[:, sl] = rng.uniform(0, P.box, size=(3, 1)) + rng.normal(0, 0.6, size=(3, sl.stop - sl.start))
    u = (np.mod(x, P.box) / P.box * TWO32).astype(np.uint64).astype(np.uint32)
    T = O.fof_threshold(P, link)
    want = brute_components(u, T)
    h, lab = O.fof(P, u, np.ones(n, np.uint32), link=link, nmin=1)
    assert np.array_equal(lab, want)
    assert len(h) == len(np.unique(want))
    assert np.array_equal(h["first"], np.unique(want))
    assert np.array_equal(h["count"], np.bincount(want)[np.unique(want)])


def test_threshold_is_inclusive():
    P = O.params(n1d=16, mesh=32, box=32.0)
    T = O.fof_threshold(P, 0.2)
    assert T == math.floor((0.2 * TWO32 / 16) ** 2)
    r = math.isqrt(T)  # r^2 <= T < (r + 1)^2
    base = 2 ** 30
    for gap, linked in ((r, True), (r + 1, False)):
        u = np.array([[base, base + gap, base + 2 * gap], [base] * 3, [base] * 3], np.uint64).astype(np.uint32)
        h, lab = O.fof(P, u, np.ones(3, np.uint32), link=0.2, nmin=1)
        assert (len(h) == 1) == linked


def test_periodic_clump_and_centre():
    P = O.params(n1d=16, mesh=32, box=32.0)
    # a symmetric cross of 7 points around x = 0 (wrapping), y = z = L/4
    s = int(0.1 * TWO32 / 16)
    c = [0, TWO32 // 4, TWO32 // 4]
    pts = [(0, 0, 0), (s, 0, 0), (-s, 0, 0), (0, s, 0), (0, -s, 0), (0, 0, s), (0, 0, -s)]
    u = np.array([[(c[a] + p[a]) % TWO32 for p in pts] for a in range(3)], np.uint64).astype(np.uint32)
    k = np.array([3, 1, 1, 2, 2, 5, 5], np.uint32)
    h, lab = O.fof(P, u, k, link=0.2, nmin=7)
    assert len(h) == 1 and h["count"][0] == 7 and h["mass"][0] == k.sum()
    assert np.allclose(h["x"][0], [0.0, 8.0, 8.0], atol=1e-12) or np.allclose(h["x"][0], [32.0, 8.0, 8.0])
    d2 = [sum(((int(u[a, i]) - 2 ** 31 + 2 ** 31) % TWO32 - 2 ** 31) ** 2 for a in range(3)) for i in range(7)]
    assert h["rmax2"][0] == max(d2)
    # nmin filters
    h2, lab2 = O.fof(P, u, k, link=0.2, nmin=8)
    assert len(h2) == 0 and np.all(lab2 == -1)


def test_mass_weighted_centre():
    P = O.params(n1d=16, mesh=32, box=32.0)
    s = int(0.05 * TWO32 / 16)
    u = np.array([[1000, 1000 + s], [2000, 2000], [3000, 3000]], np.uint64).astype(np.uint32)
    k = np.array([1, 3], np.uint32)
    h, _ = O.fof(P, u, k, link=0.2, nmin=2)
    want = (1000 + 3 * s / 4) * P.box / TWO32
    assert math.isclose(h["x"][0][0], want, rel_tol=1e-15)
