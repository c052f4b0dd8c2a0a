"""The walk's per-node decisions (Eq. 1 per walk group, the r_cut skip) pinned
on a hand-built case whose every skip / open / accept decision was derived by
hand (tests/golden/walk_open_example.json): the oracle's interaction list of
group A has exactly the hand-derived length, and its short-range force on A's
particles equals the pair sum over the hand-derived list (particles of A, B,
R, S; the three accepted monopoles; nothing of T)."""
import math

import numpy as np

import oracle as O
import walk_golden as W

TWO32 = 2 ** 32


def sorted_case():
    cs = W.case()
    P = O.params(**cs["params"])
    u, k, names = W.particles()
    _, perm = O.sort(u)
    return cs, P, u[:, perm].copy(), k[perm].copy(), names[perm]


def group_of_a(P, u, names):
    starts, counts = O.groups(P, u)
    hits = [gi for gi, (s, c) in enumerate(zip(starts, counts)) if set(names[s:s + c]) == {"A"}]
    assert len(hits) == 1, hits
    gi = hits[0]
    assert counts[gi] == 25
    return gi, int(starts[gi]), int(counts[gi])


def hand_list_force(cs, P, u, k, names, i):
    """pair sum over the hand-derived interaction list of group A, for particle i"""
    box = P.box
    n0 = P.n1d ** 3
    gm0 = 1.5 * P.omega_m * box ** 3 / (4 * math.pi * n0)
    eps0 = P.soft_frac * box / P.n1d
    rs = P.rs_cells * box / P.mesh
    rcut = P.rcut_rs * rs
    entries = []  # (lattice position, K, kmax)
    unlisted = {tuple(int(round(c / box * TWO32)) for c in pt) for pt in cs.get("unlisted_points_A", [])}
    for t in range(u.shape[1]):
        if names[t] in cs["expected_particle_clusters_A"] and tuple(int(v) for v in u[:, t]) not in unlisted:
            entries.append((u[:, t].astype(np.int64), int(k[t]), int(k[t])))
    for m in cs["expected_monopoles_A"]:
        entries.append((np.array([int(round(c / box * TWO32)) for c in m["com"]], np.int64), m["K"], m["kmax"]))
    assert len(entries) == cs["expected_list_length_A"]
    acc = np.zeros(3)
    epsi = eps0 * k[i] ** (1.0 / 3.0)
    for x, K, kmax in entries:
        d = ((x - u[:, i].astype(np.int64) + 2 ** 31) % TWO32 - 2 ** 31) * (box / TWO32)
        r = math.sqrt(float(d @ d))
        if r == 0.0 or r >= rcut:
            continue
        h = 2.8 * max(epsi, eps0 * kmax ** (1.0 / 3.0))
        acc += gm0 * K * O.pair_factor(P, r, h) * d
    return acc


def test_group_a_list_length_is_the_hand_derived_one():
    cs, P, u, k, names = sorted_case()
    gi, _, _ = group_of_a(P, u, names)
    assert O.interaction_count(P, u, k, group_index=gi) == cs["expected_list_length_A"]


def test_group_a_force_is_the_pair_sum_over_the_hand_derived_list():
    cs, P, u, k, names = sorted_case()
    _, s, c = group_of_a(P, u, names)
    g = O.accel(P, u, k, parts=2)
    for i in range(s, s + c):
        want = hand_list_force(cs, P, u, k, names, i)
        assert np.allclose(g[:, i], want, rtol=1e-12, atol=1e-12 * np.abs(want).max()), (i, g[:, i], want)


def test_hand_list_distinguishes_the_plausible_mistakes():
    """the decisions the golden pins change the force: accepting the tied node
    (or testing the cube centre) replaces two monopoles by one, skipping the
    touching leaf R drops its particles"""
    cs, P, u, k, names = sorted_case()
    _, s, _ = group_of_a(P, u, names)
    base = hand_list_force(cs, P, u, k, names, s)
    alt = dict(cs)
    alt["expected_monopoles_A"] = [cs["expected_monopoles_A"][0],
                                   {"K": 12, "com": [24.5, 20.25, 20.25], "kmax": 1}]
    alt["expected_list_length_A"] = cs["expected_list_length_A"] - 1
    assert np.abs(hand_list_force(alt, P, u, k, names, s) - base).max() > 1e-6 * np.abs(base).max()
    alt2 = dict(cs)
    alt2["expected_particle_clusters_A"] = ["A", "B", "S"]
    alt2["expected_list_length_A"] = cs["expected_list_length_A"] - 3
    alt2["unlisted_points_A"] = []
    assert np.abs(hand_list_force(alt2, P, u, k, names, s) - base).max() > 1e-3 * np.abs(base).max()
