"""Twin-run integration accuracy on the GPU (paper Sec. 3.2): the device
statistic dzs_twin_displacement against the oracle's plain definition on the
same two GPU states (exact counts), and the paper's reading of it on GPU twin
runs: lightcone particles of the runs with and without DZS stay within 8 h
(h = L / N^(1/3) / 40)."""
import numpy as np
import pytest

from oracle.displacement import twin_displacement

pytestmark = pytest.mark.gpu

EDGES = np.array([0.0, 1e-4, 1e-3, 1e-2, 0.05, 0.1, 0.2, 0.5, 1.0, 2.0, 8.0, 1e9])


@pytest.fixture(scope="module")
def dzs():
    from paper_2005_05328_gb300 import build
    build.build()
    import paper_2005_05328_gb300 as m
    m.load()
    return m


def twins(dzs, kw, steps, precision):
    a = dzs.Context(**kw, precision=precision)
    b = dzs.Context(**kw, precision=precision, dzs_on=0)
    for c in (a, b):
        c.ics()
        c.step(steps)
    return a, b


@pytest.mark.parametrize("precision", [1, 0])
def test_device_statistic_matches_the_oracle(dzs, precision):
    kw = dict(n1d=32, mesh=64, box=64.0, merge_level=2)
    a, b = twins(dzs, kw, 75, precision)
    try:
        got = dzs.dzs_twin_displacement(a.h, b.h, EDGES)
        sa, sb = a.state(), b.state()
    finally:
        a.close()
        b.close()
    want = twin_displacement(64.0, 32, sa, sb, EDGES)
    assert got[1] == want[1] > 0
    assert np.array_equal(got[0], want[0])
    assert got[2] == want[2]


@pytest.mark.parametrize("buffer_cells", [10.0, 2.0])
def test_twin_runs_displacements(dzs, buffer_cells):
    """64^3 particles in 128 Mpc/h, the lightcone sweeping the box (R from the
    box corner at z = 49 to 0 at z = 0), FP32, DZS on vs off.  Bit-identical
    until the first merge; with the paper's fiducial buffer b = 5 lambda (10
    mesh cells) every lightcone particle stays within 8 h of its twin through
    step 70 (z ~ 0.9), as in the paper's LARGEHR pair (Fig. 7, < 8 h at all z).
    Later the lightcone of this small box holds a few thousand particles, most
    in collapsed haloes whose orbits amplify the difference; those values and
    the 2-cell buffer of the benchmark configurations are reported (a thinner
    buffer lets merged particles act on lightcone particles sooner, as the
    paper's buffer scan, Fig. 9, shows)."""
    kw = dict(n1d=64, mesh=128, box=128.0, merge_level=3, seed=11, buffer_cells=buffer_cells)
    a = dzs.Context(**kw, precision=dzs.FP32)
    b = dzs.Context(**kw, precision=dzs.FP32, dzs_on=0)
    out = []
    try:
        for c in (a, b):
            c.ics()
        done = 0
        for step in (40, 70, 85, 92):
            for c in (a, b):
                c.step(step - done)
            done = step
            counts, m, mx = dzs.dzs_twin_displacement(a.h, b.h, EDGES)
            above_h = counts[8:].sum() / max(1, m)
            out.append((step, m, mx, above_h))
    finally:
        a.close()
        b.close()
    print("\nb = %g cells (step, lightcone particles, max dx/h, fraction dx > h):" % buffer_cells, out)
    assert out[0][2] == 0.0  # step 40: no merge yet in this run, twins identical
    for step, m, mx, above_h in out:
        assert m > 0
        if buffer_cells >= 10.0 and step <= 70:
            assert mx < 8.0, (step, mx)
