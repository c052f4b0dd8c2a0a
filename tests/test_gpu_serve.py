"""Serving (continuous batching of independent mocks on one GPU): requests
admitted by HBM budget in arrival order, overlapping on the device, each
result bit-identical to the same request run alone (the mix changes nothing:
separate state, deterministic reductions)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dzs():
    from paper_2005_05328_gb300 import build
    build.build()
    import paper_2005_05328_gb300 as m
    m.load()
    return m


def fnv1a(b, h=1469598103934665603):
    for x in b:
        h = ((h ^ x) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


SIZES = [(16, 32, 32.0), (32, 64, 64.0), (64, 128, 128.0)]


def mix(n, spacing):
    rng = np.random.default_rng(9)
    out = []
    for i in range(n):
        n1, m, L = SIZES[int(rng.integers(0, len(SIZES)))]
        out.append(dict(arrival_s=i * spacing, n1d=n1, mesh=m, box=L, sigma8=float(rng.uniform(0.7, 0.9)),
                        seed=int(rng.integers(1, 2 ** 31))))
    return out


def test_same_alone_and_in_mix(dzs):
    reqs = mix(10, 0.004)
    big = dzs.dzs_footprint_bytes(dzs.params(n1d=64, mesh=128, box=128.0, precision=0))
    st, wall, res = dzs.dzs_serve(reqs, hbm_budget_bytes=2.5 * big, max_active=4, steps_per_slice=8, precision=0)
    assert st == dzs.DZS_OK and all(r["status"] == 0 for r in res)
    # the mocks overlapped on the device
    ev = sorted([(r["admit_s"], 1) for r in res] + [(r["done_s"], -1) for r in res])
    conc, peak = 0, 0
    for _, d in ev:
        conc += d
        peak = max(peak, conc)
    assert peak >= 2
    for r, q in zip(res, reqs):
        assert r["admit_s"] >= q["arrival_s"] and r["done_s"] > r["admit_s"]
        assert r["records"] == q["n1d"] ** 3 and r["diag"][0] == q["n1d"] ** 3
    # each alone, through the plain API
    for r, q in zip(res, reqs):
        with dzs.Context(n1d=q["n1d"], mesh=q["mesh"], box=q["box"], sigma8=q["sigma8"], seed=q["seed"],
                         precision=0) as ctx:
            ctx.ics()
            ctx.step(96)
            rec = ctx.drain()
            n, _ = ctx.count()
            d = ctx.diagnostics()
        assert r["record_hash"] == fnv1a(rec.tobytes()), q
        assert r["n_end"] == n and r["diag"] == list(d)


def test_budget_and_oversize(dzs):
    reqs = [dict(arrival_s=0.001 * i, n1d=64, mesh=128, box=128.0, sigma8=0.8, seed=10 + i) for i in range(3)]
    small = dzs.dzs_footprint_bytes(dzs.params(n1d=64, mesh=128, box=128.0, precision=0))
    reqs.append(dict(arrival_s=0.0, n1d=128, mesh=256, box=256.0, sigma8=0.8, seed=3))  # never fits
    st, wall, res = dzs.dzs_serve(reqs, hbm_budget_bytes=1.01 * small, steps_per_slice=16, precision=0)
    assert st == dzs.DZS_ENOMEM
    assert res[-1]["status"] == dzs.DZS_ENOMEM
    assert all(r["status"] == 0 for r in res[:-1])
    # one at a time under this budget: no two admitted mocks overlap
    iv = sorted((r["admit_s"], r["done_s"]) for r in res[:-1])
    assert all(b[0] >= a[1] for a, b in zip(iv, iv[1:]))
