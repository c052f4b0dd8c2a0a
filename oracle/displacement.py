"""Oracle: particle-by-particle displacements between twin runs (paper
Sec. 3.2, integration accuracy: twin particles of the runs with and without
DZS, matched by their identity in the initial conditions, compared at the same
time; only particles inside the lightcone, since the others may be merged).

TEST INFRASTRUCTURE ONLY (see oracle.h).

Plain definition: for every id present and not crossed in both states,
    dx = |x_a - x_b| (minimum image, from the exact int32 lattice offsets),
normalised by the softening length h = L / N^(1/3) / 40 of Sec. 3.2; the
cumulative distribution of dx / h is what the paper plots.  Arithmetic in
FP64, in the order offset * (L / 2^32), squared, summed over x, y, z, square
root, divided by h.
"""
from __future__ import annotations

import numpy as np

FL_CROSSED = 1


def softening_length(box, n1d):
    """h = L / N^(1/3) / 40 (Sec. 3.2)"""
    return box / n1d / 40.0


def twin_ratios(box, n1d, st_a, st_b):
    """dx / h of every twin pair (in the id order of the pairs)"""
    in_a = (st_a["fl"] & FL_CROSSED) == 0
    in_b = (st_b["fl"] & FL_CROSSED) == 0
    ida, idb = st_a["id"][in_a], st_b["id"][in_b]
    ua, ub = st_a["u"][:, in_a], st_b["u"][:, in_b]
    common, ia, ib = np.intersect1d(ida, idb, assume_unique=True, return_indices=True)
    scale = box / 2.0 ** 32
    off = (ua[:, ia].astype(np.int64) - ub[:, ib].astype(np.int64) + 2 ** 31) % 2 ** 32 - 2 ** 31
    d = off.astype(np.float64) * scale
    s = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]
    return np.sqrt(s) / softening_length(box, n1d)


def twin_displacement(box, n1d, st_a, st_b, edges):
    """(counts per bin edges[k] <= dx/h < edges[k+1], matched pairs, max dx/h)"""
    r = twin_ratios(box, n1d, st_a, st_b)
    edges = np.asarray(edges, np.float64)
    k = np.searchsorted(edges, r, side="right") - 1
    nb = len(edges) - 1
    ok = (k >= 0) & (k < nb)
    counts = np.bincount(k[ok], minlength=nb).astype(np.uint64)
    return counts, len(r), float(r.max()) if len(r) else 0.0
