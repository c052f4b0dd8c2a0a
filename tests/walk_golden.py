"""The hand-built walk case of tests/golden/walk_open_example.json as arrays
(input construction only: no arithmetic of the method here)."""
import itertools
import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "walk_open_example.json")
T3 = (20.125, 20.25, 20.375)


def case():
    return json.load(open(GOLDEN))


def clusters():
    """name -> list of (x, y, z) in Mpc/h, as the golden file describes them"""
    c = {}
    c["A"] = [p for p in itertools.product(T3, T3, T3) if p not in ((20.375, 20.375, 20.25), (20.375, 20.375, 20.375))]
    c["B"] = list(itertools.product((20.625, 20.875), repeat=3))
    c["R"] = [(19.0, 20.25, z) for z in T3] + [(16.25, 23.75, 23.75)]
    c["S"] = [(22.5, y, z) for y in (20.125, 20.375) for z in (20.125, 20.375)]
    c["Q"] = [(x, y, z) for y in (24.25, 25.75) for x in T3 for z in (20.125, 20.375)]
    c["Q2"] = [(24.25, y, z) for y in T3 for z in T3] + [(25.25, y, 20.25) for y in T3]
    c["T"] = [(40.0, 20.25, z) for z in (20.0, 20.125, 20.25, 20.375, 20.5)]
    return c


def particles():
    """(u [3, n] uint32 lattice positions, k [n] uint32, cluster name per particle)
    in cluster order (not yet Morton-sorted)"""
    cs = case()
    box = cs["params"]["box"]
    xs, ks, names = [], [], []
    for name, pts in clusters().items():
        for p in pts:
            xs.append(p)
            ks.append(cs["clusters"][name]["k"])
            names.append(name)
    x = np.array(xs).T
    u = np.rint(x / box * 2.0 ** 32).astype(np.uint64)
    assert np.all(u.astype(np.float64) == x / box * 2.0 ** 32)  # every point sits exactly on the lattice
    return u.astype(np.uint32), np.array(ks, np.uint32), np.array(names)
