"""Pins of the oracle's dynamical DZS criterion (oracle/merge.c).

Paper Sec. 2.2.1: the dynamical opening rule (Eq. 2) with the particle
distance replaced by the node distance D_n of Eq. 3 and |a_old| by the
smallest acceleration among the particles still inside the lightcone.
Pins: alpha = 0 never merges; alpha -> infinity merges exactly the cells the
geometric rule merges in its theta -> infinity limit (D > 0 alone); the
criterion flips at the closed-form alpha* = G M l^2 / (D^4 a_min) of a
two-particle cell, with G m0 derived from the critical density; the number of
survivors is monotone in alpha; a brute-force enumeration of every cell with
the rule evaluated from its physical definition; a_min skips crossed
particles."""
import math

import numpy as np
import pytest

import oracle as O
from oracle_util import sorted_state
from test_oracle_merge import random_state

TWO32 = 2 ** 32


def g_m0(P):
    """G m0 from the critical density with H0 = 1: rho_c = 3 H0^2 / (8 pi G),
    m0 = Omega_m rho_c L^3 / N0, so G m0 = 3 Omega_m L^3 / (8 pi N0)."""
    return 3.0 * P.omega_m * P.box ** 3 / (8.0 * math.pi * P.n1d ** 3)


def blat(P):
    return int(math.floor(P.buffer_cells * TWO32 / P.mesh))


def same_state(a, b):
    return all(np.array_equal(a[f], b[f]) for f in ("u", "p", "k", "id", "fl"))


def test_amin2_skips_crossed():
    g = np.array([[3.0, 0.1, 1.0, 0.0], [4.0, 0.0, 1.0, 2.0], [0.0, 0.0, 1.0, 0.0]])
    fl = np.array([0, O.FL_CROSSED, 0, 0], np.uint8)
    assert O.amin2(g, fl) == 3.0  # |(1,1,1)|^2; the crossed (0.1,0,0) is ignored
    fl[:] = O.FL_CROSSED
    assert O.amin2(g, fl) == math.inf


def test_alpha_zero_never_merges():
    rng = np.random.default_rng(11)
    P = O.params(n1d=8, mesh=16, box=16.0, merge_level=2, criterion=1, alpha_dyn=0.0)
    st = random_state(rng, 700, P.box)
    for a2 in (1e-6, 1.0, math.inf):
        assert same_state(O.merge(P, 0, st, amin2_value=a2), st)


@pytest.mark.parametrize("rfrac", [0.0, 0.1, 0.25])
def test_alpha_infinite_is_geometric_theta_infinite(rfrac):
    """lhs is finite whenever D > 0, so alpha a_min -> infinity merges every
    cell with D > 0: the geometric rule with ceil(l / theta) = 0."""
    rng = np.random.default_rng(12)
    Pd = O.params(n1d=8, mesh=16, box=16.0, merge_level=2, buffer_cells=1.0, criterion=1, alpha_dyn=1e300)
    Pg = O.params(n1d=8, mesh=16, box=16.0, merge_level=2, buffer_cells=1.0, theta_dzs=1e300)
    st = random_state(rng, 700, Pd.box)
    rlat = int(rfrac * TWO32)
    dyn = O.merge(Pd, rlat, st, amin2_value=1.0)
    geo = O.merge(Pg, rlat, st)
    assert same_state(dyn, geo)
    assert dyn["u"].shape[1] < 700
    # no uncrossed particle: a_min = infinity, the same limit
    assert same_state(O.merge(Pd.__class__.from_buffer_copy(Pd), rlat, st, amin2_value=math.inf), geo)


def _pair_state(P, rfrac_com):
    """two unit-mass particles in one cell of side l_max (level jmin) but in
    different children, so that the jmin cell is the only candidate"""
    jmin = O.merge_jmin(P)
    side = TWO32 >> jmin
    # cell whose lower corner sits at rfrac_com of the box from the observer
    base = 2 ** 31 + int(rfrac_com * TWO32) // side * side
    q = side // 4
    u = np.array([[base + q, base + 3 * q], [base + q, base + q], [base + q, base + q]], dtype=np.uint64)
    u = (u % TWO32).astype(np.uint32)
    st = sorted_state(u, np.array([[1.0, -0.5], [0.25, 0.0], [0.0, 2.0]]), np.array([1, 1], np.uint32))
    st["fl"][:] = O.FL_CROSSED
    return st, jmin


def test_two_particle_closed_form():
    P = O.params(n1d=8, mesh=16, box=16.0, merge_level=2, buffer_cells=1.0, criterion=1)
    st, jmin = _pair_state(P, 0.3)
    rlat = int(0.05 * TWO32)
    K = 2
    com = [(2 * sum(int(v) for v in st["u"][ax]) + K) // (2 * K) for ax in range(3)]
    d = math.sqrt(sum((c - 2 ** 31) ** 2 for c in com)) * P.box / TWO32
    D = d - (rlat + blat(P)) * P.box / TWO32
    assert D > 0
    l = P.box / 2 ** jmin
    a_min = 0.37
    alpha_star = g_m0(P) * K * l ** 2 / (D ** 4 * a_min)
    for f, merged in ((1 - 1e-9, False), (1 + 1e-9, True)):
        P.alpha_dyn = alpha_star * f
        out = O.merge(P, rlat, st, amin2_value=a_min ** 2)
        assert out["u"].shape[1] == (1 if merged else 2)
        if merged:
            assert out["k"][0] == 2 and out["fl"][0] == O.FL_MERGED | O.FL_CROSSED
            assert [int(out["u"][ax, 0]) for ax in range(3)] == com
            assert np.array_equal(out["p"][:, 0], (st["p"][:, 0] + st["p"][:, 1]) / 2)
    # the same pair with its COM inside R + b never merges, whatever alpha
    P.alpha_dyn = 1e300
    out = O.merge(P, int(0.55 * TWO32), st, amin2_value=1.0)  # d_COM = 0.58 L < R + b = 0.6125 L
    assert out["u"].shape[1] == 2


def test_monotone_in_alpha():
    rng = np.random.default_rng(13)
    st = random_state(rng, 1500, 16.0)
    rlat = int(0.08 * TWO32)
    counts = []
    for alpha in (0.0, 1e-4, 1e-3, 1e-2, 0.1, 1.0, 10.0, 1e3):
        P = O.params(n1d=8, mesh=16, box=16.0, merge_level=2, buffer_cells=1.0, criterion=1, alpha_dyn=alpha)
        out = O.merge(P, rlat, st, amin2_value=1.0)
        assert out["k"].sum() == st["k"].sum()
        counts.append(out["u"].shape[1])
    assert all(b <= a for a, b in zip(counts, counts[1:]))
    assert counts[0] == 1500 and counts[-1] < counts[2] < 1500


def brute_force_dynamical(P, rlat, st, amin2):
    """Every cell with >= 2 particles at every level >= jmin, tested with
    G M l^2 / D^4 < alpha a_min (G m0 from the critical density); each
    particle takes the coarsest qualifying cell on its path."""
    u, k = st["u"], st["k"]
    n = u.shape[1]
    key = np.array([O.morton_key(*u[:, i]) for i in range(n)], dtype=np.uint64)
    jmin = O.merge_jmin(P)
    R = (rlat + blat(P)) * P.box / TWO32
    a_min = math.sqrt(amin2)
    chosen = [None] * n
    for j in range(jmin, 22):
        pref = (key >> np.uint64(3 * (21 - j))).astype(np.uint64)
        cells = {}
        for i in range(n):
            cells.setdefault(int(pref[i]), []).append(i)
        l = P.box / 2 ** j
        for members in cells.values():
            if len(members) < 2 or any(chosen[i] is not None for i in members):
                continue
            K = int(k[members].sum())
            com = [(2 * int((k[members].astype(object) * u[ax, members].astype(object)).sum()) + K) // (2 * K)
                   for ax in range(3)]
            D = math.sqrt(sum((c - 2 ** 31) ** 2 for c in com)) * P.box / TWO32 - R
            if D > 0 and g_m0(P) * K * l ** 2 / D ** 4 < P.alpha_dyn * a_min:
                for i in members:
                    chosen[i] = (j, tuple(members))
    groups, seen = [], set()
    for i in range(n):
        if chosen[i] is None:
            groups.append([i])
        elif chosen[i] not in seen:
            seen.add(chosen[i])
            groups.append(list(chosen[i][1]))
    return groups


@pytest.mark.parametrize("seed,alpha,rfrac", [(21, 0.05, 0.05), (22, 0.5, 0.15), (23, 5.0, 0.0)])
def test_brute_force_dynamical(seed, alpha, rfrac):
    rng = np.random.default_rng(seed)
    P = O.params(n1d=8, mesh=16, box=16.0, merge_level=2, buffer_cells=1.0, criterion=1, alpha_dyn=alpha)
    st = random_state(rng, 700, P.box)
    rlat = int(rfrac * TWO32)
    amin2 = 0.8
    out = O.merge(P, rlat, st, amin2_value=amin2)
    groups = brute_force_dynamical(P, rlat, st, amin2)
    assert out["u"].shape[1] == len(groups)
    assert sum(len(g) > 1 for g in groups) > 5
    for o, g in enumerate(groups):
        if len(g) == 1:
            assert out["id"][o] == st["id"][g[0]] and out["fl"][o] == st["fl"][g[0]]
        else:
            assert out["k"][o] == st["k"][g].sum() and out["id"][o] == st["id"][g].min()
