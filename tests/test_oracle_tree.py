"""Pins of the oracle short-range tree force and TreePM total (oracle/tree.c).

Paper Sec. 2.1 (monopole tree, Gaussian split), Eq. 1 (geometric opening),
Sec. 2.2 (softening ~ (M/M_init)^(1/3)).  Pins: the split identity
f_S + f_L = G m / r^2; the cubic-spline enclosed mass against direct
quadrature of the Monaghan-Lattanzio kernel; the two-body Newtonian force;
TreePM vs a direct Ewald sum (Hernquist, Bouchet & Suto 1991); the theta -> 0
walk against a brute-force pair sum; Newton's third law at theta -> 0; group
partition invariants."""
import itertools
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import erf, erfc

import oracle as O
from oracle_util import sorted_state


def test_split_identity():
    P = O.params(n1d=32, mesh=64, box=64.0)
    rs = 1.25
    for r in (0.05, 0.3, 1.0, 2.5, 5.0):
        fs = O.pair_factor(P, r, 1e-9) * r ** 3  # short-range / Newtonian
        x = r / (2 * rs)
        fl = erf(x) - 2 * x / math.sqrt(math.pi) * math.exp(-x * x)
        assert fs + fl == pytest.approx(1.0, abs=1e-15)


def spline_w(q):
    """Cubic spline kernel (Monaghan & Lattanzio 1985), support radius 1."""
    if q < 0.5:
        return 8 / math.pi * (1 - 6 * q * q + 6 * q ** 3)
    if q < 1:
        return 8 / math.pi * 2 * (1 - q) ** 3
    return 0.0


def test_spline_softening_enclosed_mass():
    """fac(r) r^3 = enclosed kernel mass within r (radius h = 1), times T(r);
    checked with T ~ 1 (r_s huge)."""
    P = O.params(n1d=32, mesh=1, box=1e6)  # r_s = 1.25e6: T = 1 to ~1e-12
    for q in (0.1, 0.3, 0.5, 0.7, 0.95, 1.0, 1.3):
        m = quad(lambda s: 4 * math.pi * s * s * spline_w(s), 0, min(q, 1.0), epsabs=1e-14)[0]
        got = O.pair_factor(P, q, 1.0) * q ** 3
        assert got == pytest.approx(m, rel=1e-9), q


def gm0(P):
    return 1.5 * P.omega_m * P.box ** 3 / (4 * math.pi * P.n1d ** 3)


@pytest.mark.parametrize("r", [0.2, 0.3, 0.45])
def test_two_body_newtonian(r):
    """Two particles at 3 eps < r < r_s / 2 in a large box: TreePM force is the
    Newtonian pull to within the PM error."""
    P = O.params(n1d=32, mesh=128, box=64.0)  # eps = 0.05, r_s = 0.625
    L = P.box
    x0 = np.array([20.3, 31.7, 40.1])
    d = np.array([0.6, -0.48, 0.64])
    x1 = x0 + r * d
    u = np.stack([x0, x1], axis=1) / L * 2 ** 32
    u = u.astype(np.uint64).astype(np.uint32)
    xr = u.astype(np.float64) * L / 2 ** 32
    sep = xr[:, 1] - xr[:, 0]
    rr = np.linalg.norm(sep)
    g = O.accel(P, u, np.ones(2, np.uint32))
    want = gm0(P) / rr ** 2
    assert np.linalg.norm(g[:, 0] - want * sep / rr) < 1e-2 * want
    assert np.linalg.norm(g[:, 1] + want * sep / rr) < 1e-2 * want


def ewald_forces(x, m, L, G=1.0):
    """Direct Ewald sum of periodic Newtonian accelerations with a neutralising
    background; alpha L = 5, real images |n| <= 2, |k| index <= 8."""
    n = x.shape[1]
    alpha = 5.0 / L
    acc = np.zeros((3, n))
    imgs = np.array(list(itertools.product(range(-2, 3), repeat=3))).T * L
    kv = np.array([v for v in itertools.product(range(-8, 9), repeat=3) if any(v)]).T * (2 * np.pi / L)
    k2 = (kv ** 2).sum(axis=0)
    kfac = 4 * np.pi / L ** 3 * np.exp(-k2 / (4 * alpha ** 2)) / k2
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            dvec = (x[:, j] - x[:, i])[:, None] + imgs
            r = np.linalg.norm(dvec, axis=0)
            f = (erfc(alpha * r) + 2 * alpha * r / math.sqrt(math.pi) * np.exp(-(alpha * r) ** 2)) / r ** 3
            acc[:, i] += G * m[j] * (dvec * f).sum(axis=1)
            ph = kv.T @ (x[:, j] - x[:, i])
            acc[:, i] += G * m[j] * (kv * (kfac * np.sin(ph))).sum(axis=1)
    return acc


def test_treepm_vs_ewald():
    rng = np.random.default_rng(11)
    P = O.params(n1d=4, mesh=64, box=16.0, soft_frac=1e-4)  # 64 particles
    n = 64
    while True:
        u = rng.integers(0, 2 ** 32, size=(3, n), dtype=np.uint64).astype(np.uint32)
        x = u.astype(np.float64) * P.box / 2 ** 32
        dd = x[:, :, None] - x[:, None, :]
        dd -= P.box * np.rint(dd / P.box)
        r = np.linalg.norm(dd, axis=0) + np.eye(n) * 1e9
        if r.min() > 0.3:
            break
    g = O.accel(P, u, np.ones(n, np.uint32))
    ge = ewald_forces(x, np.ones(n), P.box, G=gm0(P))
    err = np.linalg.norm(g - ge, axis=0) / np.linalg.norm(ge, axis=0)
    assert np.sqrt(np.mean(err ** 2)) < 0.01
    assert err.max() < 0.05


def brute_short_range(P, u, k):
    n = u.shape[1]
    L = P.box
    rs = P.rs_cells * L / P.mesh
    rcut = P.rcut_rs * rs
    eps0 = P.soft_frac * L / P.n1d
    G = gm0(P)
    g = np.zeros((3, n))
    for i in range(n):
        d = ((u.astype(np.int64) - u[:, i:i + 1].astype(np.int64) + 2 ** 31) % 2 ** 32 - 2 ** 31) * (L / 2 ** 32)
        r = np.linalg.norm(d, axis=0)
        for j in np.nonzero((r > 0) & (r < rcut))[0]:
            h = 2.8 * eps0 * max(k[i], k[j]) ** (1 / 3)
            g[:, i] += G * k[j] * O.pair_factor(P, r[j], h) * d[:, j]
    return g


def clustered_positions(rng, n, box):
    """Half uniform, half in three tight clumps (exercises deep nodes)."""
    x = rng.uniform(0, box, size=(3, n))
    for c in range(3):
        sel = slice(n // 2 + c * (n // 6), n // 2 + (c + 1) * (n // 6))
        x[:, sel] = rng.uniform(0, box, size=(3, 1)) + rng.normal(0, 0.05 * box, size=(3, n // 6))
    return (np.mod(x, box) / box * 2 ** 32).astype(np.uint64).astype(np.uint32)


def test_theta_zero_walk_is_direct_sum():
    rng = np.random.default_rng(5)
    P = O.params(n1d=8, mesh=16, box=16.0, theta=1e-12)
    u = clustered_positions(rng, 600, P.box)
    k = rng.integers(1, 9, size=600).astype(np.uint32)
    st = sorted_state(u, k=k)
    g = O.tree_accel(P, st["u"], st["k"])
    gb = brute_short_range(P, st["u"], st["k"])
    scale = np.abs(gb).max()
    assert np.allclose(g, gb, rtol=1e-12, atol=1e-12 * scale)


def test_theta_zero_newton_third_law():
    rng = np.random.default_rng(6)
    P = O.params(n1d=8, mesh=16, box=16.0, theta=1e-12)
    u = clustered_positions(rng, 900, P.box)
    k = rng.integers(1, 4, size=900).astype(np.uint32)
    st = sorted_state(u, k=k)
    g = O.tree_accel(P, st["u"], st["k"])
    tot = (g * st["k"]).sum(axis=1)
    assert np.all(np.abs(tot) < 1e-12 * (np.abs(g) * st["k"]).sum(axis=1))


def test_theta_half_close_to_direct():
    """The monopole walk at theta = 0.5 approximates the direct short-range sum
    (clustered particles: rms error of the short-range force below 2%)."""
    rng = np.random.default_rng(8)
    P = O.params(n1d=8, mesh=16, box=16.0)
    u = clustered_positions(rng, 800, P.box)
    st = sorted_state(u)
    g = O.tree_accel(P, st["u"], st["k"])
    g0 = O.tree_accel(O.params(n1d=8, mesh=16, box=16.0, theta=1e-12), st["u"], st["k"])
    err = np.linalg.norm(g - g0, axis=0)
    ref = np.linalg.norm(g0, axis=0)
    assert np.sqrt((err ** 2).mean() / (ref ** 2).mean()) < 0.02


def test_groups_partition():
    rng = np.random.default_rng(9)
    P = O.params(n1d=8, mesh=16, box=16.0)
    u = clustered_positions(rng, 3000, P.box)
    st = sorted_state(u)
    start, count = O.groups(P, st["u"])
    assert start[0] == 0
    assert np.array_equal(start[1:], start[:-1] + count[:-1])
    assert start[-1] + count[-1] == 3000
    assert np.all(count <= P.walk_group)
    # each group is the coarsest cell on its first particle's path holding
    # <= G particles (or a depth-21 leaf), i.e. its parent holds > G
    key, _ = O.sort(st["u"])
    for s, c in zip(start, count):
        for j in range(22):
            pref = int(key[s]) >> (3 * (21 - j))
            cnt = int(((key >> np.uint64(3 * (21 - j))) == pref).sum())
            if cnt <= P.walk_group or j == 21:
                break
        assert cnt == c


def test_morton_key_bits():
    # x bit b -> key bit 3b + 2, y -> 3b + 1, z -> 3b; top 21 bits of each axis
    assert O.morton_key(1 << 11, 0, 0) == 4
    assert O.morton_key(0, 1 << 11, 0) == 2
    assert O.morton_key(0, 0, 1 << 11) == 1
    assert O.morton_key(1 << 31, 0, 0) == 1 << 62
    assert O.morton_key((1 << 11) - 1, (1 << 11) - 1, (1 << 11) - 1) == 0
    assert O.morton_key(2 ** 32 - 1, 2 ** 32 - 1, 2 ** 32 - 1) == 2 ** 63 - 1


def test_sort_is_stable_and_ordered():
    rng = np.random.default_rng(10)
    u = rng.integers(0, 2 ** 32, size=(3, 1000), dtype=np.uint64).astype(np.uint32)
    u[:, 500:] = u[:, :500]  # duplicated keys
    key, perm = O.sort(u)
    ks = key[perm]
    assert np.all(np.diff(ks.astype(np.float64)) >= 0) and np.all(ks[1:] >= ks[:-1])
    # ties keep input order
    same = ks[1:] == ks[:-1]
    assert np.all(perm[1:][same] > perm[:-1][same])
    assert sorted(perm.tolist()) == list(range(1000))
