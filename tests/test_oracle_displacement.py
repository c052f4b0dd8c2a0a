"""Pins of the twin-displacement oracle (Sec. 3.2): identical runs give zero,
the minimum image crosses the periodic boundary, crossed particles are not
compared, the pairing is by id (any order), and DZS-on and DZS-off oracle runs
stay bit-identical until the first merge, then differ by small amounts."""
from fractions import Fraction
import math

import numpy as np

import oracle as O
from oracle.displacement import softening_length, twin_displacement, twin_ratios

TWO32 = 2 ** 32
EDGES = np.array([0.0, 1e-3, 1e-2, 0.1, 1.0, 8.0, 1e9])


def state(u, fl=None, ids=None):
    n = u.shape[1]
    return dict(u=np.asarray(u, np.uint32), id=np.arange(n, dtype=np.uint32) if ids is None else ids,
                fl=np.zeros(n, np.uint8) if fl is None else fl)


def test_identical_states_give_zero():
    rng = np.random.default_rng(1)
    u = rng.integers(0, TWO32, size=(3, 500), dtype=np.uint64).astype(np.uint32)
    c, m, mx = twin_displacement(64.0, 16, state(u), state(u), EDGES)
    assert m == 500 and mx == 0.0 and c[0] == 500 and c[1:].sum() == 0


def test_periodic_minimum_image_and_known_ratios():
    """particle 0: 6 lattice units across the x boundary; particle 1: a (3, 4, 0)
    lattice-unit multiple -> exact ratios from rational arithmetic"""
    box, n1d = 64.0, 16
    ua = np.array([[TWO32 - 3, 1000], [5, 2000], [7, 3000]], np.uint64).astype(np.uint32)
    q = 1 << 20
    ub = np.array([[3, 1000 + 3 * q], [5, 2000 + 4 * q], [7, 3000]], np.uint64).astype(np.uint32)
    r = twin_ratios(box, n1d, state(ua), state(ub))
    h = Fraction(64, 16 * 40)
    unit = Fraction(64, TWO32)
    want0 = 6 * unit / h
    want1 = 5 * q * unit / h  # |(3, 4, 0)| q = 5 q
    assert math.isclose(r[0], float(want0), rel_tol=1e-15)
    assert math.isclose(r[1], float(want1), rel_tol=1e-15)
    assert softening_length(box, n1d) == 0.1


def test_crossed_particles_are_not_compared_and_pairing_is_by_id():
    rng = np.random.default_rng(2)
    n = 300
    ua = rng.integers(0, TWO32, size=(3, n), dtype=np.uint64).astype(np.uint32)
    ub = (ua.astype(np.int64) + rng.integers(-5000, 5000, size=(3, n))).astype(np.uint64).astype(np.uint32)
    fa = np.zeros(n, np.uint8)
    fa[:50] = O.FL_CROSSED
    base = twin_displacement(64.0, 16, state(ua, fa), state(ub), EDGES)
    assert base[1] == n - 50
    perm = rng.permutation(n)
    sb = dict(u=ub[:, perm].copy(), id=np.arange(n, dtype=np.uint32)[perm].copy(), fl=np.zeros(n, np.uint8))
    again = twin_displacement(64.0, 16, state(ua, fa), sb, EDGES)
    assert np.array_equal(base[0], again[0]) and base[1:] == again[1:]


def test_twin_oracle_runs_identical_until_the_first_merge():
    kw = dict(n1d=8, mesh=16, box=16.0, merge_level=2)
    Pon, Poff = O.params(**kw), O.params(**kw, dzs_on=0)
    son = soff = O.initial_state(Pon)
    first_merge = None
    for step in range(96):
        son, _ = O.step(Pon, step, son)
        soff, _ = O.step(Poff, step, soff)
        c, m, mx = twin_displacement(16.0, 8, son, soff, EDGES)
        if first_merge is None:
            if son["u"].shape[1] < 8 ** 3:
                first_merge = step
            else:
                assert mx == 0.0, step  # no merge yet: bit-identical trajectories
        if step == 80:
            # after merges began: nonzero but small (the paper's LARGEHR pair keeps
            # every lightcone particle within 8 h)
            assert first_merge is not None and first_merge < 80
            assert m > 0 and 0.0 < mx < 8.0
