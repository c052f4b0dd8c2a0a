"""GPU parity tests: the CUDA path (through the C ABI) against the FP64 CPU
oracle on the same seeded inputs.

Tolerances (stated once, used below):
  - integer / index / flag work (sort order, merge membership, merged masses,
    COM lattice positions, crossing sets): bit-exact on identical input state;
  - FP64 accelerations: |dg| <= 1e-9 (|g| + 1e-3 g_rms);
  - FP32 accelerations: 99.9th percentile of |dg| / (|g| + 1e-3 g_rms) <= 1e-4;
  - FP64 time tables: 1e-13 relative; lattice radii exact;
  - drift on the lattice: |du| <= 1 unit (the FP64 product p D 2^32/L is
    rounded to the lattice on both sides; a 1-ulp difference of p or D can move
    a value across a rounding boundary).
"""
import math

import numpy as np
import pytest

import oracle as O
from kick_parity import half_step_momentum_error, momentum_bound_fp64, momentum_sum_check

pytestmark = pytest.mark.gpu

TWO32 = 2 ** 32


@pytest.fixture(scope="module")
def dzs():
    from paper_2005_05328_gb300 import build
    build.build()
    import paper_2005_05328_gb300 as m
    m.load()
    return m


C1 = dict(n1d=32, mesh=64, box=64.0, merge_level=2)
SMALL = dict(n1d=16, mesh=32, box=32.0, merge_level=2)


def oparams(**kw):
    return O.params(**{k: v for k, v in kw.items() if k not in ("precision", "device", "lc_capacity")})


_cache = {}


def oracle_run(kw, upto):
    """Oracle state after `upto` steps from its own ICs (cached per config)."""
    key = (tuple(sorted(kw.items())), upto)
    if key in _cache:
        return _cache[key]
    P = oparams(**kw)
    st = O.initial_state(P)
    for n in range(upto):
        st, _ = O.step(P, n, st)
    _cache[key] = st
    return st


def gerr(got, want):
    err = np.linalg.norm(got - want, axis=0)
    ref = np.linalg.norm(want, axis=0)
    rms = np.sqrt((ref ** 2).mean())
    return err / (ref + 1e-3 * rms)


# ---------------------------------------------------------------- tables

@pytest.mark.parametrize("kw", [C1, dict(n1d=128, mesh=256, box=256.0, merge_level=3),
                                dict(n1d=32, mesh=64, box=1024.0, rlc_mode=1, nsteps=128)])
def test_tables_match_oracle(dzs, kw):
    with dzs.Context(**kw) as ctx:
        g = ctx.tables()
    o = O.tables(oparams(**kw))
    for name in ("a", "drift", "kick1", "kick2", "rlc"):
        assert np.allclose(g[name], o[name], rtol=1e-13, atol=0), name
    assert np.array_equal(g["rlat"], o["rlat"])


# ---------------------------------------------------------------- ICs

@pytest.mark.parametrize("precision", [1, 0])
def test_ics_match_oracle(dzs, precision):
    kw = dict(SMALL, precision=precision)
    P = oparams(**kw)
    o = O.ics(P)
    with dzs.Context(**kw) as ctx:
        ctx.ics()
        s = ctx.state()
    order = np.argsort(s["id"])
    u = s["u"][:, order].astype(np.int64)
    du = (u - o["u"].astype(np.int64) + 2 ** 31) % TWO32 - 2 ** 31
    assert np.abs(du).max() <= 2
    assert (du == 0).mean() > 0.95
    pr = np.abs(s["p"][:, order] - o["p"]).max() / np.abs(o["p"]).max()
    assert pr < (1e-12 if precision == 1 else 1e-6)
    assert np.array_equal(s["k"], np.ones_like(s["k"]))
    # the ICs state is Morton-sorted
    key, perm = O.sort(s["u"])
    assert np.array_equal(perm, np.arange(len(perm)))


# ---------------------------------------------------------------- sort

def test_sort_is_the_stable_morton_order(dzs):
    rng = np.random.default_rng(3)
    kw = dict(SMALL, precision=1)
    n = 16 ** 3
    u = rng.integers(0, TWO32, size=(3, n), dtype=np.uint64).astype(np.uint32)
    u[:, 1000:1300] = u[:, 2000:2300]  # identical keys: ties keep input order
    st = dict(u=u, p=rng.normal(size=(3, n)), g=np.zeros((3, n)), k=np.ones(n, np.uint32),
              id=np.arange(n, dtype=np.uint32), fl=np.zeros(n, np.uint8))
    with dzs.Context(**kw) as ctx:
        ctx.set_state(st, 0)
        ctx.run_stages(dzs.STAGE_SORT)
        s = ctx.state()
    key, perm = O.sort(u)
    assert np.array_equal(s["id"], perm.astype(np.uint32))
    assert np.array_equal(s["u"], u[:, perm])
    assert np.array_equal(s["p"], st["p"][:, perm])


# ---------------------------------------------------------------- forces

@pytest.mark.parametrize("upto", [0, 60, 90])
@pytest.mark.parametrize("parts", [1, 2, 3])
def test_accel_fp64(dzs, upto, parts):
    st = oracle_run(SMALL, upto)
    P = oparams(**SMALL)
    want = O.accel(P, st["u"], st["k"], parts=parts)
    with dzs.Context(**dict(SMALL, precision=1)) as ctx:
        ctx.set_state(st, upto)
        got = ctx.accel(parts)
    e = gerr(got, want)
    assert e.max() <= 1e-9, (upto, parts, e.max())


@pytest.mark.parametrize("upto", [0, 60, 90])
def test_accel_fp32(dzs, upto):
    st = oracle_run(SMALL, upto)
    P = oparams(**SMALL)
    want = O.accel(P, st["u"], st["k"])
    with dzs.Context(**dict(SMALL, precision=0)) as ctx:
        ctx.set_state(st, upto)
        got = ctx.accel()
    e = gerr(got, want)
    assert np.percentile(e, 99.9) <= 1e-4, (upto, np.percentile(e, 99.9), e.max())


def test_accel_c1_fp64_all_particles(dzs):
    st = oracle_run(C1, 0)
    P = oparams(**C1)
    want = O.accel(P, st["u"], st["k"])
    with dzs.Context(**dict(C1, precision=1)) as ctx:
        ctx.set_state(st, 0)
        got = ctx.accel()
        cnt = ctx.counters()
    assert gerr(got, want).max() <= 1e-9
    assert cnt[0] > 0 and cnt[2] > 0 and cnt[3] == 0
    # the same interaction sets: evaluated (particle, entry) pairs, exactly
    assert cnt[2] == O.interaction_count(P, st["u"], st["k"])


def test_pm_mesh_delta(dzs):
    st = oracle_run(SMALL, 60)
    P = oparams(**SMALL)
    with dzs.Context(**dict(SMALL, precision=1)) as ctx:
        ctx.set_state(st, 60)
        ctx.accel(dzs.ACC_PM)
        d = ctx.mesh(dzs.MESH_DELTA)
        phi = ctx.mesh(dzs.MESH_PHI)
    want = O.cic_delta(P, st["u"], st["k"])
    assert np.allclose(d, want, rtol=0, atol=1e-12 * np.abs(want).max())
    wphi = O.pm_potential(P, want)
    assert np.allclose(phi, wphi, rtol=0, atol=1e-11 * np.abs(wphi).max())


# ---------------------------------------------------------------- merge

@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("upto,rfrac", [(70, None), (90, None), (50, 0.05), (70, 0.5), (90, 0.6)])
def test_merge_bit_exact(dzs, precision, upto, rfrac):
    """many candidates (radius from the step's table, or 0.05 L) and few
    (0.5 L, 0.6 L: ~1300 and ~300 particles beyond R + b, cells of at most a
    few dozen particles, which the first mark pass sums directly)"""
    kw = dict(SMALL, dzs_on=0)  # an un-merged evolved state
    st = oracle_run(kw, upto)
    P = oparams(**SMALL)
    rlat = int(O.tables(P)["rlat"][upto]) if rfrac is None else int(rfrac * TWO32)
    st = dict(st)
    st["fl"] = st["fl"] | O.FL_CROSSED
    if precision == 0:
        st["p"] = st["p"].astype(np.float32).astype(np.float64)
    want = O.merge(P, rlat, st)
    assert want["u"].shape[1] < st["u"].shape[1]
    with dzs.Context(**dict(SMALL, precision=precision)) as ctx:
        ctx.set_state(st, upto)
        ctx.merge_only(rlat)
        got = ctx.state()
    for name in ("u", "k", "id", "fl"):
        assert np.array_equal(got[name], want[name]), name
    if precision == 1:
        assert np.array_equal(got["p"], want["p"])
    else:
        assert np.array_equal(got["p"], want["p"].astype(np.float32).astype(np.float64))


def test_merge_nothing_qualifies_leaves_the_state(dzs):
    """radius 0.7 L: a few dozen particles lie beyond R + b, no cell qualifies;
    the state comes back unchanged, as from the oracle"""
    kw = dict(SMALL, dzs_on=0)
    st = dict(oracle_run(kw, 70))
    st["fl"] = st["fl"] | O.FL_CROSSED
    P = oparams(**SMALL)
    rlat = int(0.7 * TWO32)
    want = O.merge(P, rlat, st)
    assert want["u"].shape[1] == st["u"].shape[1]
    with dzs.Context(**dict(SMALL, precision=1)) as ctx:
        ctx.set_state(st, 70)
        before = ctx.state()
        ctx.merge_only(rlat)
        got = ctx.state()
    for name in ("u", "k", "id", "fl", "p"):
        assert np.array_equal(got[name], want[name]), name
        assert np.array_equal(got[name], before[name]), name


# ---------------------------------------------------------------- kick, drift, crossing

def test_crossing_set_bit_exact_at_rest(dzs):
    """p = g = 0: crossings decided by the lattice radii alone."""
    st = oracle_run(SMALL, 40)
    st = dict(st, p=np.zeros_like(st["p"]), g=np.zeros_like(st["g"]))
    P = oparams(**SMALL)
    tot_o, tot_g = [], []
    with dzs.Context(**dict(SMALL, precision=1)) as ctx:
        ctx.set_state(st, 40)
        so = st
        for step in range(40, 60):
            so, rec = O.kick_drift_cross(P, step, so, np.zeros_like(so["p"]))
            tot_o.append(sorted(rec["id"].tolist()))
            ctx.run_stages(dzs.STAGE_KICK_DRIFT | dzs.STAGE_CLOSE)
            r = ctx.drain()
            tot_g.append(sorted(r["id"].tolist()))
            assert tot_g[-1] == tot_o[-1], step
    assert sum(len(x) for x in tot_o) > 50


@pytest.mark.parametrize("precision", [1, 0])
def test_kick_drift_records(dzs, precision):
    st = oracle_run(SMALL, 60)
    P = oparams(**SMALL)
    if precision == 0:
        st = dict(st, p=st["p"].astype(np.float32).astype(np.float64),
                  g=st["g"].astype(np.float32).astype(np.float64))
    so, rec = O.kick_drift_cross(P, 60, st, st["g"])
    with dzs.Context(**dict(SMALL, precision=precision)) as ctx:
        ctx.set_state(st, 60)
        ctx.run_stages(dzs.STAGE_KICK_DRIFT)
        s = ctx.state()
        r = ctx.drain()
    du = (s["u"].astype(np.int64) - so["u"].astype(np.int64) + 2 ** 31) % TWO32 - 2 ** 31
    if precision == 1:
        assert np.abs(du).max() <= 1
    else:
        # FP32 kick: the kicked momentum is rounded to float (relative 2^-24 per
        # operation) before the FP64 drift product, so the lattice step can
        # differ by a few units: |du| <= 1 + 3e-7 (|p| + |g K1|) D 2^32 / L
        T = O.tables(P)
        dlat = T["drift"][60] * TWO32 / P.box
        bound = 1 + 3e-7 * (np.abs(st["p"]) + np.abs(st["g"] * T["kick1"][60])) * dlat
        assert np.all(np.abs(du) <= bound)
    assert np.array_equal(np.sort(r["id"]), np.sort(rec["id"]))
    assert np.array_equal(s["fl"], so["fl"])
    # the opening kick of every particle (not only the crossing ones):
    # p_{n+1/2} = p_n + K(a_n, a_{n+1/2}) g_n; FP32 rounds p, g K1 and the sum
    K1 = O.tables(P)["kick1"][60]
    scale = np.abs(st["p"]) + np.abs(st["g"]) * K1
    ptol = 1e-13 if precision == 1 else 3e-7
    assert np.all(np.abs(s["p"] - so["p"]) <= ptol * scale + 1e-300), np.abs(s["p"] - so["p"]).max()
    ro, rg = rec[np.argsort(rec["id"])], r[np.argsort(r["id"])]
    tol = 1e-12 if precision == 1 else 1e-6
    assert np.allclose(rg["a_cross"], ro["a_cross"], rtol=tol)
    assert np.allclose(rg["x"], ro["x"], rtol=0, atol=tol * P.box)
    assert np.allclose(rg["p"], ro["p"], rtol=tol, atol=tol * np.abs(ro["p"]).max())


# ---------------------------------------------------------------- full step

@pytest.mark.parametrize("upto", [20, 75])
def test_full_step_fp64(dzs, upto):
    st = oracle_run(SMALL, upto)
    P = oparams(**SMALL)
    so, rec = O.step(P, upto, st)
    with dzs.Context(**dict(SMALL, precision=1)) as ctx:
        ctx.set_state(st, upto)
        ctx.step(1)
        s = ctx.state()
        r = ctx.drain()
        d = ctx.diagnostics()
    assert np.array_equal(np.sort(r["id"]), np.sort(rec["id"]))
    assert np.array_equal(s["id"], so["id"]) and np.array_equal(s["k"], so["k"])
    du = (s["u"].astype(np.int64) - so["u"].astype(np.int64) + 2 ** 31) % TWO32 - 2 ** 31
    assert np.abs(du).max() <= 1
    assert gerr(s["g"], so["g"]).max() <= 1e-6
    # momenta after the closing kick: the half-step momenta agree to rounding,
    # the full momenta within rounding + K2 |dg|
    assert half_step_momentum_error(P, upto, s, so).max() <= 1e-12
    ok, worst = momentum_bound_fp64(P, upto, s, so)
    assert ok, worst
    od = O.diagnostics(P, so["u"], so["p"], so["k"])
    assert d[0] == od[0] and d[7] == od[7]
    assert np.allclose(d[4:7], od[4:7], rtol=1e-12)
    assert momentum_sum_check(d, s, so, P) == (True, True)


@pytest.mark.parametrize("upto", [20, 75])
def test_full_step_fp32(dzs, upto):
    """FP32 state and forces: the oracle steps the FP32-rounded state; merge
    membership, masses and ids agree exactly, accelerations within the FP32
    bound, half-step momenta within a few float roundings"""
    st = oracle_run(SMALL, upto)
    st = dict(st, p=st["p"].astype(np.float32).astype(np.float64), g=st["g"].astype(np.float32).astype(np.float64))
    P = oparams(**SMALL)
    so, rec = O.step(P, upto, st)
    with dzs.Context(**dict(SMALL, precision=0)) as ctx:
        ctx.set_state(st, upto)
        ctx.step(1)
        s = ctx.state()
        r = ctx.drain()
        d = ctx.diagnostics()
    assert np.array_equal(np.sort(r["id"]), np.sort(rec["id"]))
    assert np.array_equal(s["id"], so["id"]) and np.array_equal(s["k"], so["k"])
    assert np.percentile(gerr(s["g"], so["g"]), 99.9) <= 1e-4
    assert half_step_momentum_error(P, upto, s, so).max() <= 2e-6
    od = O.diagnostics(P, so["u"], so["p"], so["k"])
    assert d[0] == od[0] and d[7] == od[7]
    own, _ = momentum_sum_check(d, s, so, P)
    assert own


def test_steps_are_deterministic(dzs):
    st = oracle_run(SMALL, 70)
    outs = []
    for _ in range(2):
        with dzs.Context(**dict(SMALL, precision=0)) as ctx:
            ctx.set_state(st, 70)
            ctx.step(5)
            outs.append((ctx.state(), ctx.drain()))
    (a, ra), (b, rb) = outs
    for name in a:
        assert np.array_equal(a[name], b[name]), name
    assert ra.tobytes() == rb.tobytes()


def test_full_run_records_every_particle_once(dzs):
    kw = dict(SMALL, precision=0)
    with dzs.Context(**kw) as ctx:
        ctx.ics()
        done = ctx.step(200)
        rec = ctx.drain()
        n, step = ctx.count()
        d = ctx.diagnostics()
    assert done == 96 and step == 96
    assert sorted(rec["id"].tolist()) == list(range(16 ** 3))
    assert d[0] == 16 ** 3  # mass conserved through every merge
    assert n < 16 ** 3  # DZS merged particles outside the lightcone


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("upto", [0, 80])
def test_accel_coarse_mesh(dzs, precision, upto):
    """mesh spacing twice the particle spacing (as the 512^3 configuration):
    r_cut = 11.25 Mpc/h spans many walk groups, so the walk evaluates its lists
    in the single range-guarded pass; parity as in the other force tests"""
    kw = dict(n1d=16, mesh=16, box=32.0, merge_level=2)
    st = oracle_run(kw, upto)
    P = oparams(**kw)
    want = O.accel(P, st["u"], st["k"])
    with dzs.Context(**dict(kw, precision=precision)) as ctx:
        ctx.set_state(st, upto)
        got = ctx.accel()
        cnt = ctx.counters()
    e = gerr(got, want)
    if precision == 1:
        assert e.max() <= 1e-9, e.max()
        assert cnt[2] == O.interaction_count(P, st["u"], st["k"])
    else:
        assert np.percentile(e, 99.9) <= 1e-4, np.percentile(e, 99.9)
