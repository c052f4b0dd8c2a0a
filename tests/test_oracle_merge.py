"""Pins of the oracle DZS merge (oracle/merge.c).

Paper Sec. 2.2 (top-down walk, Fig. 2; centre-of-mass transfer), Eq. 3 (node
distance D_n = max(d - R_lc - b, 0)), Sec. 2.2.1 (l_n / D_n < theta_dzs,
l_max).  Pins: exact mass conservation, bounded COM rounding, momentum
conservation; no merge inside R_lc + b; every member of a merged cell lies
beyond R_lc + b for theta_dzs <= 1/sqrt(3); the (lambda / l_max)^3 floor on
an unperturbed lattice (the analogue of the Table 2 floor, Sec. 3.3); a
brute-force enumeration of all cells; the hand-built walk of Fig. 2."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from oracle_util import lattice_positions, sorted_state

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TWO32 = 2 ** 32


def d2_obs(u):
    """exact squared distance to the observer at 2^31 (Python integers)"""
    off = (u.astype(np.int64) - 2 ** 31).astype(object)
    return (off ** 2).sum(axis=0)


def random_state(rng, n, box, clump=True):
    x = rng.uniform(0, box, size=(3, n))
    if clump:
        m = n // 8
        for c in range(4):
            x[:, c * m:(c + 1) * m] = rng.uniform(0, box, size=(3, 1)) + rng.normal(0, 0.03 * box, size=(3, m))
    u = (np.mod(x, box) / box * TWO32).astype(np.uint64).astype(np.uint32)
    p = rng.normal(size=(3, n))
    k = rng.integers(1, 5, size=n).astype(np.uint32)
    st = sorted_state(u, p, k)
    st["fl"][:] = O.FL_CROSSED
    st["id"] = rng.permutation(n).astype(np.uint32)[np.argsort(np.argsort(st["id"]))]
    return st


def test_conservation_and_buffer():
    rng = np.random.default_rng(1)
    P = O.params(n1d=16, mesh=32, box=32.0, merge_level=3)
    st = random_state(rng, 4096, P.box)
    rlat = int(0.2 * TWO32)
    out = O.merge(P, rlat, st)
    assert out["u"].shape[1] < 4096
    assert out["k"].sum() == st["k"].sum()
    merged = out["fl"] & O.FL_MERGED > 0
    kk = out["k"][merged].astype(np.int64)
    S0 = (st["u"].astype(np.int64) * st["k"]).sum(axis=1)
    S1 = (out["u"].astype(np.int64) * out["k"]).sum(axis=1)
    assert np.all(np.abs(S1 - S0) <= kk.sum() / 2)
    P0 = (st["p"] * st["k"]).sum(axis=1)
    P1 = (out["p"] * out["k"]).sum(axis=1)
    assert np.allclose(P1, P0, rtol=0, atol=1e-13 * np.abs(st["p"] * st["k"]).sum())
    # particles within R + b are untouched
    blat = int(2.0 * TWO32 / 32)
    inside = np.array([d <= (rlat + blat) ** 2 for d in d2_obs(st["u"])])
    ids_in = set(st["id"][inside].tolist())
    out_ids = {i: j for j, i in enumerate(out["id"].tolist())}
    for t in np.nonzero(inside)[0]:
        j = out_ids[st["id"][t]]
        assert not merged[j]
        assert np.array_equal(out["u"][:, j], st["u"][:, t]) and np.array_equal(out["p"][:, j], st["p"][:, t])
    assert len(ids_in) == inside.sum()
    # survivors keep Morton order
    key, perm = O.sort(out["u"])
    assert np.array_equal(perm, np.arange(out["u"].shape[1]))


def test_threshold_definition():
    P = O.params(n1d=32, mesh=64, box=64.0)
    rlat = 123456789
    blat = 2 * TWO32 // 64
    for j in (4, 5, 8, 12, 21):
        t = O.merge_threshold(P, rlat, j)
        assert abs(t - (rlat + blat + 2 ** (32 - j) / 0.1)) < 2
    assert O.merge_threshold(P, rlat, 1) >= TWO32  # 10 L / 2 never fits
    assert O.merge_jmin(P) == 4  # l_max = 2 lambda = 4 Mpc/h = 64 / 2^4
    assert O.merge_jmin(O.params(n1d=48, box=96.0, merge_level=3)) == 4  # 96/16 = 6 <= 8
    assert O.merge_jmin(O.params(n1d=128, box=256.0, merge_level=3)) == 5


@pytest.mark.parametrize("ell,ratio", [(2, 8), (3, 64)])
def test_unperturbed_lattice_floor(ell, ratio):
    """R_lc = 0, b = 0, theta_dzs = inf: every l_max cell merges, leaving
    N (lambda / l_max)^3 particles (no cell COM sits on the observer)."""
    P = O.params(n1d=16, mesh=32, box=32.0, merge_level=ell, theta_dzs=math.inf, buffer_cells=0.0)
    u = lattice_positions(16, 32.0)
    st = sorted_state(u)
    out = O.merge(P, 0, st)
    assert out["u"].shape[1] == 16 ** 3 // ratio
    assert np.all(out["k"] == ratio)


@pytest.mark.parametrize("theta", [0.1, 0.5])
def test_members_beyond_buffer(theta):
    """theta_dzs <= 1/sqrt(3): every member of a merged cell lies beyond
    R_lc + b (member distance >= d_COM - sqrt(3) l > R + b)."""
    rng = np.random.default_rng(3)
    P = O.params(n1d=16, mesh=32, box=32.0, merge_level=3, theta_dzs=theta)
    st = random_state(rng, 3000, P.box)
    rlat = int(0.15 * TWO32)
    blat = int(2.0 * TWO32 / 32)
    groups = brute_force_groups(P, rlat, st)
    for g in groups:
        if len(g) > 1:
            assert all(d > (rlat + blat) ** 2 for d in d2_obs(st["u"][:, g]))


def brute_force_groups(P, rlat, st):
    """Enumerate every cell with >= 2 particles at every level >= jmin, test
    it, and give each particle the coarsest qualifying cell on its path."""
    u, k = st["u"], st["k"]
    n = u.shape[1]
    key = np.array([O.morton_key(*u[:, i]) for i in range(n)], dtype=np.uint64)
    jmin = O.merge_jmin(P)
    chosen = [None] * n
    for j in range(jmin, 22):
        pref = (key >> np.uint64(3 * (21 - j))).astype(np.uint64)
        cells = {}
        for i in range(n):
            cells.setdefault(int(pref[i]), []).append(i)
        T = O.merge_threshold(P, rlat, j)
        for members in cells.values():
            if len(members) < 2 or T >= TWO32:
                continue
            if any(chosen[i] is not None for i in members):
                continue
            K = int(k[members].sum())
            com = [(2 * int((k[members].astype(object) * u[ax, members].astype(object)).sum()) + K) // (2 * K)
                   for ax in range(3)]
            d2 = sum((c - 2 ** 31) ** 2 for c in com)
            if d2 > T * T:
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


@pytest.mark.parametrize("seed,theta,rfrac", [(4, 0.1, 0.1), (5, 0.5, 0.2), (6, 0.3, 0.0)])
def test_brute_force_cells(seed, theta, rfrac):
    rng = np.random.default_rng(seed)
    P = O.params(n1d=8, mesh=16, box=16.0, merge_level=2, theta_dzs=theta, buffer_cells=1.0)
    st = random_state(rng, 700, P.box)
    rlat = int(rfrac * TWO32)
    out = O.merge(P, rlat, st)
    groups = brute_force_groups(P, rlat, st)
    assert out["u"].shape[1] == len(groups)
    assert sum(len(g) > 1 for g in groups) > 5
    for o, g in enumerate(groups):
        if len(g) == 1:
            i = g[0]
            assert np.array_equal(out["u"][:, o], st["u"][:, i])
            assert np.array_equal(out["p"][:, o], st["p"][:, i])
            assert out["k"][o] == st["k"][i] and out["id"][o] == st["id"][i] and out["fl"][o] == st["fl"][i]
        else:
            K = int(st["k"][g].sum())
            assert out["k"][o] == K
            assert out["id"][o] == st["id"][g].min()
            assert out["fl"][o] == O.FL_MERGED | O.FL_CROSSED
            for ax in range(3):
                S = sum(int(st["k"][i]) * int(st["u"][ax, i]) for i in g)
                assert out["u"][ax, o] == (2 * S + K) // (2 * K)
                acc = 0.0
                for i in g:  # left-to-right FP64 sum in Morton order
                    acc = acc + float(st["k"][i]) * float(st["p"][ax, i])
                assert out["p"][ax, o] == acc / K


def test_fig2_walk_example():
    case = json.load(open(os.path.join(GOLDEN, "merge_walk_example.json")))
    P = O.params(**case["params"])
    names = list(case["positions"])
    x = np.array([case["positions"][nm] for nm in names]).T
    u = (x / P.box * TWO32).astype(np.uint64).astype(np.uint32)
    st = sorted_state(u, np.zeros((3, len(names))), np.ones(len(names), np.uint32))
    st["fl"][:] = O.FL_CROSSED
    rlat = int(case["rlc"] / P.box * TWO32)
    out = O.merge(P, rlat, st)
    got = []
    ids = st["id"]  # original index in `names`
    for o in range(out["u"].shape[1]):
        if out["fl"][o] & O.FL_MERGED:
            # members: the particles whose ids fall in this merged cell
            members = [names[int(i)] for i in ids if int(i) >= 0]
            got.append(("merged", int(out["k"][o]), names[int(out["id"][o])]))
        else:
            got.append(("kept", 1, names[int(out["id"][o])]))
    want = []
    for g in case["expected_groups"]:
        if len(g) == 1:
            want.append(("kept", 1, g[0]))
        else:
            want.append(("merged", len(g), min(g, key=lambda nm: names.index(nm))))
    assert sorted(got) == sorted(want)
