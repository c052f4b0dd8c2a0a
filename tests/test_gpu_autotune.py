"""The autotuner's knobs are execution-only: the two walk evaluation modes give
bit-identical states (same pairs, same order), the serving loop's thread and
slice counts give bit-identical mocks; the tuner picks a valid mode and caches
it."""
import json
import os

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


@pytest.mark.parametrize("kw", [dict(n1d=32, mesh=64, box=64.0, merge_level=2),
                                dict(n1d=32, mesh=32, box=64.0, merge_level=2)])
@pytest.mark.parametrize("precision", [0, 1])
def test_walk_modes_are_bit_identical(dzs, kw, precision):
    out = []
    for mode in (dzs.WALK_MASKED, dzs.WALK_GUARDED, dzs.WALK_AUTO):
        with dzs.Context(**kw, precision=precision, walk_eval=mode) as ctx:
            ctx.ics()
            ctx.step(6)
            out.append((ctx.state(), ctx.drain()))
    (a, ra) = out[0]
    for b, rb in out[1:]:
        for key in a:
            assert np.array_equal(a[key], b[key]), key
        assert ra.tobytes() == rb.tobytes()


def test_serving_knobs_do_not_change_results(dzs):
    reqs = [dict(arrival_s=0.0, n1d=n, mesh=2 * n, box=2.0 * n, sigma8=0.8, seed=77 + i)
            for i, n in enumerate((16, 32, 16, 32, 16, 16))]
    res = []
    for th, sl in ((1, 96), (4, 3), (8, 8)):
        st, _, r = dzs.dzs_serve(reqs, hbm_budget_bytes=150e9, steps_per_slice=sl, host_threads=th,
                                 precision=dzs.FP32)
        assert st == dzs.DZS_OK
        res.append([(x["record_hash"], x["n_end"], x["records"], tuple(x["diag"])) for x in r])
    assert res[0] == res[1] == res[2]


def test_tuner_picks_and_caches(dzs, tmp_path, monkeypatch):
    from paper_2005_05328_gb300 import autotune
    monkeypatch.setenv("DZS_TUNE_CACHE", str(tmp_path / "tune.json"))
    mode = autotune.tune_walk(32, 64, 64.0, dzs.FP32)
    assert mode in (dzs.WALK_MASKED, dzs.WALK_GUARDED)
    db = json.load(open(tmp_path / "tune.json"))
    (key, entry), = db.items()
    assert entry["walk_eval"] == mode and len(entry["ms"]) == 2
    assert autotune.tune_walk(32, 64, 64.0, dzs.FP32) == mode  # from the cache
    P = autotune.tuned_params(n1d=32, mesh=64, box=64.0, precision=dzs.FP32)
    assert P.walk_eval == mode and P.walk_group == 32 and P.leaf_bucket == 8


def test_batch_api_results_equal_solo_runs(dzs):
    """dzs_batch_*: six mocks of four sizes stepped together by worker threads
    (each on its own stream) end bit-identical to the same mocks stepped alone"""
    import torch
    shapes = [(16, 32, 5), (32, 64, 6), (24, 48, 7), (16, 32, 8), (32, 64, 9), (48, 96, 10)]
    solo = []
    for n1, m, seed in shapes:
        with dzs.Context(n1d=n1, mesh=m, box=2.0 * n1, seed=seed, precision=dzs.FP32) as ctx:
            ctx.ics()
            ctx.step(40)
            solo.append((ctx.state(), ctx.drain()))
    streams = [torch.cuda.Stream() for _ in shapes]
    ctxs = [dzs.Context(n1d=n1, mesh=m, box=2.0 * n1, seed=seed, precision=dzs.FP32, stream=s.cuda_stream)
            for (n1, m, seed), s in zip(shapes, streams)]
    try:
        for c in ctxs:
            c.ics()
        with dzs.Batch(ctxs, host_threads=3) as b:
            done = b.step(25, slice=4)
            assert list(done) == [25] * len(ctxs)
            done = b.step(15, slice=7)
            assert list(done) == [15] * len(ctxs)
            b.synchronize()
        for c, (st, rec) in zip(ctxs, solo):
            s2 = c.state()
            for key in st:
                assert np.array_equal(s2[key], st[key]), key
            assert c.drain().tobytes() == rec.tobytes()
    finally:
        for c in ctxs:
            c.close()
