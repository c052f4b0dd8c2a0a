"""Pins of the oracle KDK step, lightcone crossing and diagnostics
(oracle/step.c).

Paper Sec. 2.1 (global steps), Sec. 1 footnote and Sec. 3.1.3 (particles are
written to the lightcone as it sweeps them; R_lc is the comoving distance).
Pins: linear growth of a small Zel'dovich plane wave follows D+(a) (force
normalisation, kick/drift factors and IC momenta together); every particle
that starts inside R_lc is recorded exactly once by a = 1 (R_lc(1) = 0); the
crossing time of a particle at rest solves d = R_lc(a*) on the step's linear
interpolation; PHYSICAL mode flags particles outside R_lc at the start; exact
mass conservation over a DZS run."""
import math

import numpy as np
import pytest

import oracle as O
from oracle_util import lattice_positions, sorted_state

TWO32 = 2 ** 32


def plane_wave_state(P, amp_frac):
    n1d, box = P.n1d, P.box
    ai = 1 / (1 + P.z_init)
    A = amp_frac * box / (2 * math.pi) / O.growth(P, ai)
    q = lattice_positions(n1d, box).astype(np.float64) * box / TWO32
    disp = np.zeros((3, n1d ** 3))
    disp[0] = O.growth(P, ai) * A * np.sin(2 * math.pi * q[0] / box)
    u = lattice_positions(n1d, box, disp)
    pf = ai ** 2 * O.hubble_e(P, ai) * O.growth_rate(P, ai)
    p = np.zeros((3, n1d ** 3))
    p[0] = pf * disp[0]
    st = sorted_state(u, p)
    st["g"] = O.accel(P, st["u"], st["k"])
    return st, q, A


def test_linear_growth_plane_wave():
    P = O.params(n1d=8, mesh=16, box=16.0, dzs_on=0, theta=1e-9)
    st, q, A = plane_wave_state(P, 0.001)
    T = O.tables(P)
    worst_x = worst_p = 0.0
    for n in range(P.nsteps):
        st, _ = O.step(P, n, st)
        if n % 6 == 5:
            a = T["a"][n + 1]
            qq = q[:, st["id"]]
            s = np.sin(2 * math.pi * qq[0] / P.box)
            x = st["u"][0].astype(np.float64) * P.box / TWO32
            dx = (x - qq[0] + P.box / 2) % P.box - P.box / 2
            amp = (dx * s).sum() / (s * s).sum()
            pamp = (st["p"][0] * s).sum() / (s * s).sum()
            D = O.growth(P, a)
            plin = a ** 2 * O.hubble_e(P, a) * O.growth_rate(P, a) * D * A
            worst_x = max(worst_x, abs(amp / (D * A) - 1))
            worst_p = max(worst_p, abs(pamp / plin - 1))
            # transverse axes stay on the lattice
            assert np.array_equal(st["u"][1:], lattice_positions(P.n1d, P.box)[1:, st["id"]])
    assert worst_x < 3e-3
    assert worst_p < 5e-3


def test_every_particle_crosses_once():
    P = O.params(n1d=8, mesh=16, box=16.0, nsteps=48, dzs_on=0)
    st = O.initial_state(P)
    seen = []
    T = O.tables(P)
    for n in range(P.nsteps):
        st, rec = O.step(P, n, st)
        seen.extend(rec["id"].tolist())
        assert np.all(rec["a_cross"] >= T["a"][n] - 1e-15) and np.all(rec["a_cross"] <= T["a"][n + 1] + 1e-15)
        # the record sits on the interpolated lightcone: |x* - o| = R_n + t (R_n+1 - R_n)
        t = (rec["a_cross"] - T["a"][n]) / (T["a"][n + 1] - T["a"][n])
        rlin = T["rlc"][n] + t * (T["rlc"][n + 1] - T["rlc"][n])
        d = np.linalg.norm(rec["x"] - P.box / 2, axis=1)
        # (|x| along the step's straight path is convex: its chord error is
        # second order in the step's displacement)
        assert np.all(np.abs(d - rlin) < 5e-3 * P.box / P.n1d)
    assert sorted(seen) == list(range(P.n1d ** 3))
    assert np.all(st["fl"] & O.FL_CROSSED)


def test_particle_at_rest_crossing_time():
    P = O.params(n1d=8, mesh=16, box=16.0, nsteps=16)
    T = O.tables(P)
    n = 9
    d = 0.5 * (T["rlc"][n] + T["rlc"][n + 1]) + 0.1 * (T["rlc"][n] - T["rlc"][n + 1])
    off = int(d / math.sqrt(3) / P.box * TWO32)
    u = np.array([[2 ** 31 + off], [2 ** 31 + off], [2 ** 31 + off]], np.uint32)
    st = dict(u=u, p=np.zeros((3, 1)), k=np.ones(1, np.uint32), id=np.array([7], np.uint32),
              fl=np.zeros(1, np.uint8))
    for m in range(n):
        st, rec = O.kick_drift_cross(P, m, st, np.zeros((3, 1)))
        assert len(rec) == 0
    st, rec = O.kick_drift_cross(P, n, st, np.zeros((3, 1)))
    assert len(rec) == 1 and rec["id"][0] == 7 and st["fl"][0] & O.FL_CROSSED
    dl = math.sqrt(3) * off * P.box / TWO32
    t = (T["rlc"][n] - dl) / (T["rlc"][n] - T["rlc"][n + 1])
    assert rec["a_cross"][0] == pytest.approx(T["a"][n] + t * (T["a"][n + 1] - T["a"][n]), rel=1e-13)
    st, rec = O.kick_drift_cross(P, n + 1, st, np.zeros((3, 1)))
    assert len(rec) == 0  # recorded once only


def test_physical_mode_initial_flags():
    P = O.params(n1d=8, mesh=16, box=4000.0, rlc_mode=1)  # chi(z=49) >> box
    T = O.tables(P)
    assert T["rlc"][0] == pytest.approx(math.sqrt(3) * 2000.0, rel=1e-15)
    P2 = O.params(n1d=8, mesh=16, box=16000.0, rlc_mode=1)
    T2 = O.tables(P2)
    u = lattice_positions(8, 16000.0)
    fl = O.initial_flags(P2, u, np.zeros(512, np.uint8))
    x = u.astype(np.float64) * 16000.0 / TWO32 - 8000.0
    d = np.linalg.norm(x, axis=0)
    assert np.array_equal(fl & 1 > 0, d >= T2["rlat"][0] * 16000.0 / TWO32 - 1e-6)
    assert 0 < fl.sum() < 512


def test_dzs_run_conserves_mass_and_merges():
    P = O.params(n1d=8, mesh=16, box=16.0, nsteps=24, merge_level=2)
    st = O.initial_state(P)
    for n in range(P.nsteps):
        st, _ = O.step(P, n, st)
        d = O.diagnostics(P, st["u"], st["p"], st["k"])
        assert d[0] == 512 and d[7] == st["u"].shape[1]
    assert st["u"].shape[1] < 512
    assert np.all(st["k"][st["fl"] & O.FL_MERGED > 0] > 1)
    ids = st["id"]
    assert len(set(ids.tolist())) == len(ids)
