"""The batched configuration's instance shapes (N1 in {32, 48, 64, 96}, L =
2 N1 Mpc/h, mesh 2 N1: meshes of 3 2^a points and 48^3 / 96^3 particle
lattices) through the CUDA path against the oracle, and the 64-mock batch run
through the serving loop with every mock checked against the same mock run
alone.  Tolerances as in test_gpu_parity.py."""
import numpy as np
import pytest

import oracle as O
from kick_parity import half_step_momentum_error, momentum_bound_fp64, momentum_sum_check

pytestmark = pytest.mark.gpu

TWO32 = 2 ** 32
C48 = dict(n1d=48, mesh=96, box=96.0, merge_level=3, seed=1003)
C24 = dict(n1d=24, mesh=48, box=48.0, merge_level=2, seed=7)


@pytest.fixture(scope="module")
def dzs():
    from paper_2005_05328_gb300 import build
    build.build()
    import paper_2005_05328_gb300 as m
    m.load()
    return m


def oparams(**kw):
    return O.params(**{k: v for k, v in kw.items() if k not in ("precision",)})


def gerr(got, want):
    err = np.linalg.norm(got - want, axis=0)
    ref = np.linalg.norm(want, axis=0)
    rms = np.sqrt((ref ** 2).mean())
    return err / (ref + 1e-3 * rms)


_cache = {}


def evolved(kw, upto):
    key = (tuple(sorted(kw.items())), upto)
    if key not in _cache:
        P = oparams(**kw)
        st = O.initial_state(P)
        for n in range(upto):
            st, _ = O.step(P, n, st)
        _cache[key] = st
    return _cache[key]


@pytest.mark.parametrize("kw", [C48, C24])
@pytest.mark.parametrize("precision", [1, 0])
def test_ics_3x2a_lattice(dzs, kw, precision):
    P = oparams(**kw)
    o = O.ics(P)
    with dzs.Context(**kw, precision=precision) as ctx:
        ctx.ics()
        s = ctx.state()
    order = np.argsort(s["id"])
    du = (s["u"][:, order].astype(np.int64) - o["u"].astype(np.int64) + 2 ** 31) % TWO32 - 2 ** 31
    assert np.abs(du).max() <= 2 and (du == 0).mean() > 0.95
    pr = np.abs(s["p"][:, order] - o["p"]).max() / np.abs(o["p"]).max()
    assert pr < (1e-12 if precision == 1 else 1e-6)


def test_pm_mesh_3x2a(dzs):
    st = evolved(C24, 40)
    P = oparams(**C24)
    with dzs.Context(**C24, precision=1) as ctx:
        ctx.set_state(st, 40)
        ctx.accel(dzs.ACC_PM)
        d = ctx.mesh(dzs.MESH_DELTA)
        phi = ctx.mesh(dzs.MESH_PHI)
    want = O.cic_delta(P, st["u"], st["k"])
    assert np.allclose(d, want, rtol=0, atol=1e-12 * np.abs(want).max())
    wphi = O.pm_potential(P, want)
    assert np.allclose(phi, wphi, rtol=0, atol=1e-11 * np.abs(wphi).max())


@pytest.mark.parametrize("upto", [0, 40])
def test_accel_3x2a(dzs, upto):
    st = evolved(C24, upto)
    P = oparams(**C24)
    want = O.accel(P, st["u"], st["k"])
    for precision in (1, 0):
        with dzs.Context(**C24, precision=precision) as ctx:
            ctx.set_state(st, upto)
            got = ctx.accel()
        e = gerr(got, want)
        if precision == 1:
            assert e.max() <= 1e-9, e.max()
        else:
            assert np.percentile(e, 99.9) <= 1e-4, np.percentile(e, 99.9)


def test_full_step_3x2a_fp64(dzs):
    st = evolved(C24, 50)
    P = oparams(**C24)
    so, rec = O.step(P, 50, st)
    with dzs.Context(**C24, precision=1) as ctx:
        ctx.set_state(st, 50)
        ctx.step(1)
        s = ctx.state()
        r = ctx.drain()
        d = ctx.diagnostics()
    assert np.array_equal(np.sort(r["id"]), np.sort(rec["id"]))
    assert np.array_equal(s["id"], so["id"]) and np.array_equal(s["k"], so["k"])
    du = (s["u"].astype(np.int64) - so["u"].astype(np.int64) + 2 ** 31) % TWO32 - 2 ** 31
    assert np.abs(du).max() <= 1
    assert gerr(s["g"], so["g"]).max() <= 1e-6
    assert half_step_momentum_error(P, 50, s, so).max() <= 1e-12
    ok, worst = momentum_bound_fp64(P, 50, s, so)
    assert ok, worst
    assert momentum_sum_check(d, s, so, P) == (True, True)


def splitmix64(state):
    state = (state + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return state, z ^ (z >> 31)


def batch_requests():
    """64 mocks: 16 each of N1 = 32, 48, 64, 96; L = 2 N1, mesh 2 N1; seeds
    1000 + i; sigma8_i = 0.7 + 0.2 U_i with U from SplitMix64(4242)"""
    st, out = 4242, []
    for i in range(64):
        st, z = splitmix64(st)
        n1 = (32, 48, 64, 96)[i % 4]
        out.append(dict(arrival_s=0.0, n1d=n1, mesh=2 * n1, box=2.0 * n1, sigma8=0.7 + 0.2 * (z >> 11) / 2.0 ** 53,
                        seed=1000 + i))
    return out


def fnv1a(b, h=1469598103934665603):
    for x in b:
        h = ((h ^ x) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def test_batch_of_64_same_alone_and_in_mix(dzs):
    reqs = batch_requests()
    st, wall, res = dzs.dzs_serve(reqs, hbm_budget_bytes=150e9, steps_per_slice=8, precision=dzs.FP32)
    assert st == dzs.DZS_OK and all(r["status"] == 0 for r in res)
    work = sum(q["n1d"] ** 3 * 96 for q in reqs)
    print("\nbatch of 64: %.2f s, %.3e particle-steps/s, %.0f mocks/h" % (wall, work / wall, 64 * 3600 / wall))
    for i in (0, 1, 2, 3, 61, 62):  # one of each size, and two more
        q = reqs[i]
        with dzs.Context(n1d=q["n1d"], mesh=q["mesh"], box=q["box"], sigma8=q["sigma8"], seed=q["seed"],
                         precision=dzs.FP32) as ctx:
            ctx.ics()
            ctx.step(96)
            rec = ctx.drain()
            d = ctx.diagnostics()
        assert res[i]["record_hash"] == fnv1a(rec.tobytes()), q
        assert res[i]["diag"] == list(d)
        assert res[i]["records"] == q["n1d"] ** 3
