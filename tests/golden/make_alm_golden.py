"""Write tests/golden/alm_nside256_seed5.json: spherical-harmonic coefficients
a_lm (Sec. 3.1.2, the angular power spectrum of the lightcone sky map) of the
oracle's Nside = 256 sky map of 2,000,000 seeded records, for degrees above
the range of scipy's sph_harm_y (the oracle then evaluates Y_lm with mpmath,
which GPU test hosts may lack).  Calls only oracle/.  Run from the repo
root: python tests/golden/make_alm_golden.py"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from oracle import sht  # noqa: E402
from observe_inputs import random_records  # noqa: E402

NSIDE, SEED, N, BOX = 256, 5, 2_000_000, 32.0
PAIRS = [(650, 0), (700, 350), (767, 0), (767, 1), (767, 383), (767, 766), (767, 767), (720, 100)]


def main():
    P = O.params(n1d=16, mesh=32, box=BOX)
    rec = random_records(SEED, N, BOX)
    m = O.skymap(P, rec, NSIDE)
    ang = sht.pixel_angles(NSIDE)
    om = m.astype(np.float64)
    out = {"cite": "Sec. 3.1.2 (Fig. 4): angular power spectrum of the lightcone sky map",
           "nside": NSIDE, "seed": SEED, "n_records": N, "box": BOX,
           "map_sha256": hashlib.sha256(m.tobytes()).hexdigest(), "map_sum": int(m.sum()),
           "alm": []}
    for l, mm in PAIRS:
        a = sht.alm_one(om, NSIDE, l, mm, ang)
        out["alm"].append([l, mm, a.real, a.imag])
    with open(os.path.join(HERE, "alm_nside256_seed5.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
