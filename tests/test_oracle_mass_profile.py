"""The mean particle mass as a function of the distance from the observer
(Sec. 3, the showcase figure of the small twin runs at z = 0.05): structures
inside the lightcone are untouched by DZS, and outside it the mean mass does
not rise at once beyond R_lc + b (the geometric criterion merges only cells
small in angle as seen from the buffer surface), then grows with distance,
noisily (a merged particle carries the mass of its cell, large in clusters,
small in voids).  Oracle runs (FP64): 16^3 and 32^3 boxes to a = 1/1.05.

Pins: every particle within R_lc(a) + b has k = 1; sum k = N0; the run without
DZS has k = 1 everywhere; the mean multiplicity per distance bin beyond
R_lc + b rises with distance (Spearman rank correlation > 0.6) and exceeds 1.5
in the outer half of the occupied radii."""
import numpy as np
import pytest
from scipy.stats import spearmanr

import oracle as O

TWO32 = 2 ** 32


def run_to(P, a_target):
    T = O.tables(P)
    st = O.initial_state(P)
    n = 0
    while T["a"][n] < a_target:
        st, _ = O.step(P, n, st)
        n += 1
    return st, T["rlc"][n]


def distances(P, u):
    off = u.astype(np.int64) - 2 ** 31
    return np.sqrt((off.astype(float) ** 2).sum(axis=0)) * P.box / TWO32


def mass_profile(d, k, nbins=12):
    edges = np.linspace(0.0, d.max() * (1 + 1e-12), nbins + 1)
    mid, mean = [], []
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (d >= lo) & (d < hi)
        if sel.sum() >= 5:
            mid.append(0.5 * (lo + hi))
            mean.append(k[sel].mean())
    return np.array(mid), np.array(mean)


@pytest.mark.parametrize("kw", [dict(n1d=16, mesh=32, box=32.0, merge_level=2),
                                dict(n1d=32, mesh=64, box=64.0, merge_level=3)])
def test_mean_mass_profile(kw):
    P = O.params(**kw)
    st, rlc = run_to(P, 1 / 1.05)
    d, k = distances(P, st["u"]), st["k"].astype(float)
    b = P.buffer_cells * P.box / P.mesh
    assert st["k"].sum() == P.n1d ** 3
    assert np.all(k[d < rlc + b] == 1)
    mid, mean = mass_profile(d, k)
    out = mid > rlc + b
    rho = spearmanr(mid[out], mean[out]).correlation
    assert rho > 0.6, (mid, mean)
    assert mean[mid > 0.5 * d.max()].mean() > 1.5
    # the twin run without DZS keeps every particle at m0
    Ps = O.params(**kw, dzs_on=0)
    ss, _ = run_to(Ps, 1 / 1.05)
    assert np.all(ss["k"] == 1) and ss["u"].shape[1] == P.n1d ** 3
