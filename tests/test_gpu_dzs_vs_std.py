"""DZS-on vs DZS-off statistics through the CUDA path (Sec. 3.1.2-3.1.3: the
sky-projected lightcone, its angular power spectrum and the 3D lightcone of
twin runs agree to ~0.1%).  Statistical, not parity: the two runs differ by
design outside the lightcone, and FP32 trajectories diverge chaotically.
Twin runs from the same seeded ICs, FP32 forces, the paper's geometric
criterion (theta_dzs = 0.1), SWEEP lightcone; observables over the whole
run.  The measured values are printed (pytest -s) and bounded below.
Measured on GB300 (N_end/N0; sky-map L1 relative difference at Nside 64; 3D
lightcone L1 at 64^3; median |C_l ratio - 1| for l <= 128; raw P(k) at the
fundamental mode, z = 0):
  64^3, L = 128:  0.119; 6.8e-4; 2.1e-4; 1.7e-3; +0.9%
  128^3, L = 256: 0.032; 1.7e-3; 3.0e-4; 2.4e-3; +0.2%
The paper quotes <= 0.1% per pixel at Nside 256 for runs with far more
particles per pixel."""
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


def twin(dzs, kw, nside, mesh_lc, nbins):
    out = {}
    for on in (0, 1):
        with dzs.Context(**kw, dzs_on=on, precision=0) as ctx:
            ctx.observe(nside=nside, mesh=mesh_lc, a_lo=0.0, a_hi=2.0)
            ctx.ics()
            ctx.step(kw.get("nsteps", 96))
            rec = ctx.drain()
            out[on] = dict(n=ctx.count()[0], mass=int(rec["k"].sum()), sky=ctx.skymap(nside).astype(float),
                           grid=ctx.lcdensity(mesh_lc).astype(float), cl=ctx.skymap_alm(2 * nside)[0],
                           pk=ctx.power_spectrum(nbins, shot=False))
    return out[0], out[1]


@pytest.mark.parametrize("kw,bound_sky,bound_grid,bound_cl", [
    (dict(n1d=64, mesh=128, box=128.0, merge_level=3, seed=4), 2e-3, 2e-3, 1e-2),
    (dict(n1d=128, mesh=256, box=256.0, merge_level=3, seed=2), 2e-3, 2e-3, 1e-2),
])
def test_twin_runs(dzs, kw, bound_sky, bound_grid, bound_cl):
    nside, mesh_lc = 64, 64
    lmax_pk = kw["n1d"] // 8  # k < pi / l_max with l_max = 4 lambda
    a, b = twin(dzs, kw, nside, mesh_lc, lmax_pk)
    n0 = kw["n1d"] ** 3
    assert a["mass"] == b["mass"] == n0
    assert b["n"] < 0.5 * a["n"]
    sky = np.abs(a["sky"] - b["sky"]).sum() / a["sky"].sum()
    grid = np.abs(a["grid"] - b["grid"]).sum() / a["grid"].sum()
    cl = np.abs(b["cl"][1:] / a["cl"][1:] - 1)
    pk = b["pk"][1] / a["pk"][1] - 1
    print("\n%s: N_end/N0 %.4f; sky L1 %.2e; 3D L1 %.2e; C_l |rel| median %.2e max %.2e; "
          "P(k<pi/l_max) rel %s" % (kw, b["n"] / n0, sky, grid, np.median(cl), cl.max(), np.round(pk, 4)))
    assert sky <= bound_sky
    assert grid <= bound_grid
    assert np.median(cl) <= bound_cl
    # the final-time P(k) at the two largest scales, where merged particles
    # still carry the large-scale mass distribution (the paper avoids P(k) of
    # the de-refined volume)
    assert np.all(np.abs(pk[:2]) <= 2e-2), pk[:2]


def lightcone_halos(dzs, kw, on, cadence=4, start=24):
    """Sec. 3.1.1: FoF catalogues every `cadence` steps; a halo enters the
    lightcone catalogue when all its members are inside R_lc at the output
    (rmax2 < R_lat^2) and its centre lies in the shell the lightcone sweeps
    before the next output (piecewise-constant approximation)."""
    masses = []
    with dzs.Context(**kw, dzs_on=on, precision=0) as ctx:
        T = ctx.tables()
        rlc, rlat = T["rlc"], T["rlat"]
        ctx.ics()
        ctx.step(start)
        step = start
        half = kw["box"] / 2
        while step < 96:
            h = ctx.fof(link=0.2, nmin=20)
            nxt = min(step + cadence, 96)
            d = np.sqrt(((h["x"] - half) ** 2).sum(axis=1))
            sel = (h["rmax2"] < int(rlat[step]) ** 2) & (d < rlc[step]) & (d >= rlc[nxt])
            masses.append(h["mass"][sel])
            ctx.step(nxt - step)
            step = nxt
    return np.concatenate(masses)


def test_lightcone_halo_mass_function(dzs):
    """the paper's LCHMF comparison (Fig. 3: sub-percent): twin 128^3 runs
    (the bench workload), FoF every 2 steps from step 30, haloes of >= 20
    particles.  Measured on GB300: 156 haloes (std) vs 159 (DZS), total mass
    7586 vs 7600 m0 (+0.2%); per mass bin [16, 32, 64, 128, 256, 512):
    77/52/19/6/1/1 vs 87/45/19/6/1/1"""
    kw = dict(n1d=128, mesh=256, box=256.0, merge_level=3, seed=2)
    a = lightcone_halos(dzs, kw, 0, cadence=2, start=30)
    b = lightcone_halos(dzs, kw, 1, cadence=2, start=30)
    bins = 2.0 ** np.arange(4, 16)
    ha, _ = np.histogram(a, bins)
    hb, _ = np.histogram(b, bins)
    print("\nLCHMF std %s\nLCHMF dzs %s  (haloes %d vs %d, mass %d vs %d)" % (ha, hb, len(a), len(b), a.sum(), b.sum()))
    assert len(a) > 50
    assert abs(len(b) - len(a)) <= max(3, 0.05 * len(a))
    assert abs(int(b.sum()) - int(a.sum())) <= 0.05 * a.sum()


def test_mean_mass_profile(dzs):
    """the showcase figure's bottom panels (Sec. 3, z = 0.05): mean particle
    mass against the distance from the observer in twin 64^3 runs (L = 128,
    FP32 forces).  DZS leaves every particle within R_lc + b at m0 and the
    mean mass rises outside, with noise; the run without DZS stays at m0.
    Measured on GB300 (R_lc = 1.64, b = 2 Mpc/h), mean k per twelfth of the
    radial range from the centre: 1.02, 1.22, 1.78, 2.1, 3.3, 7.9, 8.8, 11.3,
    14.0, 25.0, 56.8, 58.8."""
    from scipy.stats import spearmanr
    kw = dict(n1d=64, mesh=128, box=128.0, merge_level=3, seed=4)
    out = {}
    for on in (0, 1):
        with dzs.Context(**kw, dzs_on=on, precision=0) as ctx:
            T = ctx.tables()
            n = int(np.argmax(T["a"] >= 1 / 1.05))
            ctx.ics()
            ctx.step(n)
            st = ctx.state()
            out[on] = (st, T["rlc"][n])
    std, _ = out[0]
    assert np.all(std["k"] == 1) and std["u"].shape[1] == 64 ** 3
    st, rlc = out[1]
    off = st["u"].astype(np.int64) - 2 ** 31
    d = np.sqrt((off.astype(float) ** 2).sum(axis=0)) * kw["box"] / 2 ** 32
    k = st["k"].astype(float)
    b = 2.0 * kw["box"] / kw["mesh"]  # buffer of 2 PM cells
    assert st["k"].sum() == 64 ** 3
    assert np.all(k[d < rlc + b] == 1)
    edges = np.linspace(0.0, d.max() * (1 + 1e-12), 13)
    mid = 0.5 * (edges[:-1] + edges[1:])
    mean = np.array([k[(d >= lo) & (d < hi)].mean() if ((d >= lo) & (d < hi)).sum() >= 5 else np.nan
                     for lo, hi in zip(edges[:-1], edges[1:])])
    ok = np.isfinite(mean) & (mid > rlc + b)
    print("\nmean k per radial bin (R_lc %.2f, b %.1f): %s" % (rlc, b, np.round(mean, 2)))
    assert spearmanr(mid[ok], mean[ok]).correlation > 0.6
    assert np.nanmean(mean[mid > 0.5 * d.max()]) > 1.5
