"""Autotuner for the execution-only knobs of the library (never the physics:
the walk group bound G, the leaf size B, theta, the mesh and every other
parameter that changes a result stay as given).

Knobs:
  - walk_eval: how the tree walk evaluates its interaction lists (a range-test
    pass then force arithmetic for the pairs within r_cut, or one guarded
    pass).  Both evaluate the same pairs in the same order, so results are
    identical; only the time differs, with the group size against r_cut and
    with clustering.
  - host_threads, steps_per_slice of the serving loop (dzs_serve): how many
    host threads issue the mocks' kernels and how many steps each slice
    enqueues.

Measurements use the library's own CUDA-event stage timers (walk) or the
serving loop's wall clock, on the GPU the process uses.  Results are cached
in a JSON file keyed by the GPU name and the workload shape:
$DZS_TUNE_CACHE, else ~/.cache/dzs_gb300/tuning.json.
"""
from __future__ import annotations

import json
import os
import time

from . import WALK_GUARDED, WALK_MASKED, Context, dzs_serve, params


def cache_path() -> str:
    p = os.environ.get("DZS_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "dzs_gb300", "tuning.json")


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(db: dict) -> None:
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass  # a read-only home: tuning still applies to this process


def _gpu_name(device: int) -> str:
    import torch
    return torch.cuda.get_device_name(device)


def _walk_ms(p, warm_steps: int, steps: int) -> float:
    """walk milliseconds per step over `steps` steps after `warm_steps` from the ICs"""
    with Context(p) as ctx:
        ctx.ics()
        ctx.step(warm_steps)
        ctx.set_profiling(True)
        done = ctx.step(steps)
        prof = ctx.profile()
    return prof["walk"][0] / max(1, done)


def tune_walk(n1d: int, mesh: int, box: float, precision: int = 0, device: int = 0, force: bool = False,
              **physics) -> int:
    """Best walk_eval for this workload shape (cached).  The candidates are
    timed over a few steps early in the run (near-uniform, where the list
    evaluation matters most) and a few steps late (clustered)."""
    key = "walk|%s|n1d=%d|mesh=%d|box=%g|prec=%d|%s" % (_gpu_name(device), n1d, mesh, box, precision,
                                                     ",".join("%s=%s" % kv for kv in sorted(physics.items())))
    db = _load()
    if not force and key in db:
        return int(db[key]["walk_eval"])
    base = dict(n1d=n1d, mesh=mesh, box=box, precision=precision, device=device, **physics)
    nst = params(**base).nsteps
    timings = {}
    for mode in (WALK_MASKED, WALK_GUARDED):
        p = params(**base, walk_eval=mode)
        timings[mode] = _walk_ms(p, 2, 3) + _walk_ms(p, int(0.8 * nst), 3)
    best = min(timings, key=timings.get)
    db[key] = {"walk_eval": int(best), "ms": {str(k): v for k, v in timings.items()}, "when": time.time()}
    _store(db)
    return int(best)


def tuned_params(**kw):
    """params(**kw) with walk_eval chosen by tune_walk (unless given)"""
    if "walk_eval" not in kw:
        physics = {k: v for k, v in kw.items() if k not in ("n1d", "mesh", "box", "precision", "device", "seed",
                                                             "sigma8", "lc_capacity", "capacity")}
        kw = dict(kw, walk_eval=tune_walk(kw["n1d"], kw["mesh"], kw["box"], kw.get("precision", 0),
                                          kw.get("device", 0), **physics))
    return params(**kw)


def tune_serving(requests, hbm_budget_bytes: float, device: int = 0, force: bool = False,
                 threads=(4, 8, 16), slices=(4, 8, 16), **base):
    """Best (host_threads, steps_per_slice) for a request mix (cached by the
    mix's sizes); each candidate serves the whole sample once."""
    sizes = sorted({(int(r["n1d"]), int(r["mesh"])) for r in requests})
    key = "serve|%s|n=%d|sizes=%s|%s" % (_gpu_name(device), len(requests), sizes,
                                         ",".join("%s=%s" % kv for kv in sorted(base.items())))
    db = _load()
    if not force and key in db:
        return int(db[key]["host_threads"]), int(db[key]["steps_per_slice"])
    walls = {}
    for th in threads:
        for sl in slices:
            st, wall, _ = dzs_serve(requests, hbm_budget_bytes=hbm_budget_bytes, steps_per_slice=sl,
                                    host_threads=th, device=device, **base)
            if st == 0:
                walls[(th, sl)] = wall
    best = min(walls, key=walls.get)
    db[key] = {"host_threads": best[0], "steps_per_slice": best[1],
               "wall_s": {"%d,%d" % k: v for k, v in walls.items()}, "when": time.time()}
    _store(db)
    return best
