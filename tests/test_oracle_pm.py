"""Pins of the oracle particle-mesh force (oracle/pm.c).

Paper Sec. 2.1: the PM part solves Poisson's equation on a mesh in Fourier
space, joined to the tree with an exponential (Gaussian) kernel.  Pins: CIC
mass conservation, node-exact deposit, translation covariance, momentum
conservation of the symmetric deposit/interpolation pair, and the force of an
isolated particle against the analytic long-range pair force
    f_L(r) = G m / r^2 [erf(r / 2 r_s) - r / (r_s sqrt(pi)) exp(-r^2 / 4 r_s^2)]."""
import math

import numpy as np
import pytest
from scipy.special import erf

import oracle as O


def rand_u(rng, n):
    return rng.integers(0, 2 ** 32, size=(3, n), dtype=np.uint64).astype(np.uint32)


def test_cic_mass_conservation():
    rng = np.random.default_rng(1)
    P = O.params(n1d=16, mesh=32, box=32.0)
    u = rand_u(rng, 5000)
    k = rng.integers(1, 9, size=5000).astype(np.uint32)
    d = O.cic_delta(P, u, k)
    nbar = 16 ** 3 / 32 ** 3
    assert ((d + 1) * nbar).sum() == pytest.approx(k.sum(), rel=1e-13)


def test_cic_particle_on_node():
    P = O.params(n1d=16, mesh=32, box=32.0)
    node = np.array([3, 17, 31])
    u = (node.astype(np.uint64) << np.uint64(27)).astype(np.uint32).reshape(3, 1)
    d = O.cic_delta(P, u, np.array([5], np.uint32))
    nbar = 16 ** 3 / 32 ** 3
    n = (d + 1) * nbar
    assert n[3, 17, 31] == pytest.approx(5.0, rel=1e-15)
    n[3, 17, 31] = 0
    assert np.abs(n).max() < 1e-12


def test_cic_split_between_nodes():
    P = O.params(n1d=16, mesh=32, box=32.0)
    # one quarter of a cell past node 5 along y, on nodes along x and z
    u = np.array([[2 << 27], [(5 << 27) + (1 << 25)], [7 << 27]], np.uint64).astype(np.uint32)
    n = (O.cic_delta(P, u, np.array([1], np.uint32)) + 1) * (16 ** 3 / 32 ** 3)
    assert n[2, 5, 7] == pytest.approx(0.75, abs=1e-14)
    assert n[2, 6, 7] == pytest.approx(0.25, abs=1e-14)


def test_cic_translation_covariance():
    rng = np.random.default_rng(2)
    P = O.params(n1d=16, mesh=32, box=32.0)
    u = rand_u(rng, 2000)
    k = np.ones(2000, np.uint32)
    d0 = O.cic_delta(P, u, k)
    u1 = u.copy()
    u1[1] = (u1[1].astype(np.uint64) + (3 << 27)) % (1 << 32)
    d1 = O.cic_delta(P, u1, k)
    assert np.allclose(d1, np.roll(d0, 3, axis=1), rtol=0, atol=1e-12)


def test_pm_momentum_conservation():
    """Same CIC weights for deposit and interpolation and an antisymmetric
    stencil: sum_i k_i g_i = 0 to rounding."""
    rng = np.random.default_rng(3)
    P = O.params(n1d=16, mesh=32, box=32.0)
    u = rand_u(rng, 3000)
    k = rng.integers(1, 5, size=3000).astype(np.uint32)
    phi = O.pm_potential(P, O.cic_delta(P, u, k))
    g = O.pm_accel(P, phi, u)
    tot = (g * k).sum(axis=1)
    assert np.all(np.abs(tot) < 1e-11 * (np.abs(g) * k).sum(axis=1))


def test_pm_isolated_particle_long_range_force():
    P = O.params(n1d=32, mesh=128, box=64.0)
    M, L = P.mesh, P.box
    dx = L / M
    rs = 1.25 * dx
    gm0 = 1.5 * 0.3 * L ** 3 / (4 * math.pi * 32 ** 3)
    src = np.array([[int(0.37 * 2 ** 32)], [int(0.61 * 2 ** 32)], [int(0.13 * 2 ** 32)]], np.uint32)
    phi = O.pm_potential(P, O.cic_delta(P, src, np.ones(1, np.uint32)))
    rng = np.random.default_rng(0)
    r = np.geomspace(2 * dx, L / 16, 60)
    dirs = rng.normal(size=(3, r.size))
    dirs /= np.linalg.norm(dirs, axis=0)
    xs = src.astype(np.float64) * L / 2 ** 32
    u = (np.mod(xs + dirs * r, L) / L * 2 ** 32).astype(np.uint64).astype(np.uint32)
    g = O.pm_accel(P, phi, u)
    x = r / (2 * rs)
    fl = gm0 / r ** 2 * (erf(x) - 2 * x / math.sqrt(math.pi) * np.exp(-x * x))
    fn = gm0 / r ** 2
    radial = -(g * dirs).sum(axis=0)  # toward the source
    tangential = np.linalg.norm(g + dirs * radial, axis=0)
    err = (radial - fl) / fn
    assert np.sqrt(np.mean(err ** 2)) < 0.01
    assert np.abs(err).max() < 0.03
    assert np.sqrt(np.mean((tangential / fn) ** 2)) < 0.01
