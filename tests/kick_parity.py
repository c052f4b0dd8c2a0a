"""Momentum checks of the fused kicks against the oracle (test helpers).

The closing half-kick of a KDK step (Sec. 2.1, global steps) sets
p_{n+1} = p_{n+1/2} + K(a_{n+1/2}, a_{n+1}) g_{n+1}.  Positions after the
drift may differ from the oracle's by a lattice unit, which moves g_{n+1} by
up to ~1e-6 relative; the half-step momentum p_{n+1/2} = p_{n+1} - K2 g_{n+1}
does not depend on that, so both sides' half-step momenta are compared, which
pins the kick factor (a wrong table index or half-step changes it by percents)
and the merged momenta Sum k p / K (Sec. 2.2: merges conserve momentum).
"""
import numpy as np

import oracle as O


def half_step_momentum_error(P, step, s, so):
    """|(p - K2 g)_gpu - (p - K2 g)_oracle| / (|p| + K2 |g| + 1e-3 rms), per
    particle (max over axes); s and so must hold the same particles in the
    same order"""
    K2 = O.tables(P)["kick2"][step]
    ph_g = s["p"] - K2 * s["g"]
    ph_o = so["p"] - K2 * so["g"]
    scale = np.abs(so["p"]) + K2 * np.abs(so["g"])
    rms = np.sqrt((scale ** 2).mean())
    return (np.abs(ph_g - ph_o) / (scale + 1e-3 * rms)).max(axis=0)


def momentum_bound_fp64(P, step, s, so):
    """FP64: |p_gpu - p_oracle| <= 1e-12 (|p| + K2|g|) + K2 |g_gpu - g_oracle|"""
    K2 = O.tables(P)["kick2"][step]
    dp = np.abs(s["p"] - so["p"])
    scale = np.abs(so["p"]) + K2 * np.abs(so["g"])
    bound = 1e-12 * (scale + 1e-3 * np.sqrt((scale ** 2).mean())) + K2 * np.abs(s["g"] - so["g"]) * (1 + 1e-9)
    return bool(np.all(dp <= bound)), float((dp - bound).max())


def momentum_sum_check(d, s, so, P, rel=1e-12):
    """The FP64 diagnostic Sum k p (d[1:4]): equal to the oracle's diagnostic of
    the GPU's own state at `rel` of Sum k |p| (the reduction itself), and
    within Sum k |p_gpu - p_oracle| (+ the same rounding) of the oracle state's
    (triangle inequality)"""
    own = O.diagnostics(P, s["u"], s["p"], s["k"])
    scale = float((s["k"][None, :] * np.abs(s["p"])).sum(axis=1).max())
    ok_own = np.all(np.abs(d[1:4] - own[1:4]) <= rel * scale)
    od = O.diagnostics(P, so["u"], so["p"], so["k"])
    spread = (s["k"][None, :] * np.abs(s["p"] - so["p"])).sum(axis=1)
    ok_or = np.all(np.abs(d[1:4] - od[1:4]) <= spread + 2 * rel * scale)
    return bool(ok_own), bool(ok_or)
