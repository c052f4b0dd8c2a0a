"""Helpers shared by the oracle tests (no arithmetic of the method here)."""
import numpy as np

import oracle as O


def lattice_positions(n1d, box, disp=None):
    """Unperturbed lattice q = i L / n1d (plus an optional displacement in Mpc/h),
    as uint32 SoA [3, n] in id order."""
    i = np.arange(n1d)
    q = (i.astype(np.uint64) << np.uint64(32)) // np.uint64(n1d)
    qa, qb, qc = np.meshgrid(q, q, q, indexing="ij")
    u = np.stack([qa.ravel(), qb.ravel(), qc.ravel()]).astype(np.uint64)
    if disp is not None:
        du = np.rint(disp * (2.0 ** 32 / box)).astype(np.int64)
        u = (u.astype(np.int64) + du) % (1 << 32)
    return u.astype(np.uint32)


def x_of(u, box):
    return u.astype(np.float64) * (box / 2.0 ** 32)


def sorted_state(u, p=None, k=None):
    n = u.shape[1]
    key, perm = O.sort(u)
    st = dict(u=u[:, perm].copy(),
              p=(np.zeros((3, n)) if p is None else p[:, perm].copy()),
              k=(np.ones(n, np.uint32) if k is None else k[perm].copy()),
              id=perm.astype(np.uint32), fl=np.zeros(n, np.uint8))
    return st
