"""Seeded synthetic lightcone records for the observable tests (an input
generator only: no arithmetic of the method).  Directions uniform in the
box around the observer, multiplicities 1..8, crossing expansion factors
uniform in [0.02, 1)."""
import numpy as np

RECORD_DTYPE = np.dtype([("id", "<u4"), ("k", "<u4"), ("a_cross", "<f8"),
                         ("x", "<f8", (3,)), ("p", "<f8", (3,))])


def random_records(seed, n, box, a=(0.02, 1.0)):
    rng = np.random.default_rng(seed)
    rec = np.zeros(n, RECORD_DTYPE)
    rec["id"] = np.arange(n)
    rec["k"] = rng.integers(1, 9, size=n)
    rec["a_cross"] = rng.uniform(*a, size=n)
    rec["x"] = rng.uniform(0, box, size=(n, 3))
    return rec
