"""Pins of the oracle's lightcone observables (oracle/observe.c, oracle/sht.py).

Paper Sec. 3.1.2: lightcone mass projected on an equal-area sky pixelisation
(Górski et al. 2005, RING order) and its angular power spectrum.  Pins: the
12 base pixels of Nside = 1 at their textbook centres; every pixel centre maps
back to its own pixel; ring sizes and latitudes of the scheme; equal areas by
Monte Carlo (chi^2 of uniform directions) and a bound on the distance of a
direction to its pixel centre; known pixels of the axes; the sky map keeps
the record mass and honours the a* window; the harmonic analysis returns the
closed-form coefficients of a constant, a dipole and single-harmonic maps."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import sht


def test_base_pixels_nside1():
    z, phi = O.pix2zphi(1, np.arange(12))
    q = np.pi / 4
    assert np.allclose(z, [2 / 3] * 4 + [0] * 4 + [-2 / 3] * 4, atol=1e-15)
    want = [q, 3 * q, 5 * q, 7 * q, 0, 2 * q, 4 * q, 6 * q, q, 3 * q, 5 * q, 7 * q]
    assert np.allclose(phi, want, atol=1e-15)


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 16, 64, 256])
def test_centres_round_trip(nside):
    pix = np.arange(12 * nside * nside)
    assert np.array_equal(O.ang2pix(nside, O.pix2vec(nside, pix)), pix)


@pytest.mark.parametrize("nside", [1, 4, 32])
def test_ring_structure(nside):
    npix = 12 * nside * nside
    rings = np.array([O.pix2ring(nside, p)[0] for p in range(npix)])
    z, phi = O.pix2zphi(nside, np.arange(npix))
    assert rings.min() == 1 and rings.max() == 4 * nside - 1
    assert np.all(np.diff(rings) >= 0)  # RING order runs north to south
    for i in range(1, 4 * nside):
        sel = rings == i
        size = 4 * min(i, nside, 4 * nside - i)
        assert sel.sum() == size
        zi = z[sel]
        assert np.all(zi == zi[0])
        if i < nside:
            assert math.isclose(zi[0], 1 - i * i / (3 * nside * nside), rel_tol=0, abs_tol=1e-15)
        elif i <= 3 * nside:
            assert math.isclose(zi[0], 4 / 3 - 2 * i / (3 * nside), rel_tol=0, abs_tol=1e-15)
        # equally spaced in phi, increasing
        d = np.diff(phi[sel])
        assert np.allclose(d, 2 * np.pi / size, rtol=1e-13)


def test_axes():
    for nside in (1, 2, 256, 1024):
        npix = 12 * nside * nside
        assert O.ang2pix(nside, np.array([0.0, 0.0, 1.0])) == 0
        assert O.ang2pix(nside, np.array([0.0, 0.0, -1.0])) == npix - 4
        eq = npix // 2 - 2 * nside  # first pixel of the equatorial ring 2 nside
        assert O.ang2pix(nside, np.array([1.0, 0.0, 0.0])) == eq
        assert O.ang2pix(nside, np.array([0.0, 1.0, 0.0])) == eq + nside
        assert O.ang2pix(nside, np.array([-1.0, 0.0, 0.0])) == eq + 2 * nside
        assert O.ang2pix(nside, np.array([0.0, 0.0, 0.0])) == 0


@pytest.mark.parametrize("nside", [2, 4, 16])
def test_equal_area_and_locality(nside):
    rng = np.random.default_rng(7)
    n = 2_000_000
    v = rng.normal(size=(3, n))
    pix = O.ang2pix(nside, v)
    npix = 12 * nside * nside
    cnt = np.bincount(pix, minlength=npix)
    mean = n / npix
    from scipy.stats import chi2
    stat = ((cnt - mean) ** 2 / mean).sum()
    p = chi2.sf(stat, npix - 1)
    assert 1e-5 < p < 1 - 1e-5
    assert np.abs(cnt - mean).max() < 5.5 * math.sqrt(mean)
    # every direction lies within ~ one pixel size of its pixel centre
    c = O.pix2vec(nside, pix[:200_000])
    u = v[:, :200_000] / np.linalg.norm(v[:, :200_000], axis=0)
    ang = np.arccos(np.clip((c * u).sum(axis=0), -1, 1))
    assert ang.max() < 1.5 * math.sqrt(4 * math.pi / npix)


def test_skymap_mass_and_window():
    P = O.params(n1d=8, mesh=16, box=16.0)
    rng = np.random.default_rng(3)
    rec = np.zeros(5000, O.RECORD_DTYPE)
    rec["k"] = rng.integers(1, 9, size=5000)
    rec["a_cross"] = rng.uniform(0.02, 1.0, size=5000)
    rec["x"] = rng.uniform(0, 16.0, size=(5000, 3))
    rec["x"][0] = 8.0  # at the observer: direction +z
    rec["a_cross"][0] = 0.5
    m = O.skymap(P, rec, 8)
    assert m.sum() == rec["k"].sum() and m[0] >= rec["k"][0]
    lo, hi = 0.3, 0.7
    mw = O.skymap(P, rec, 8, lo, hi)
    inw = (rec["a_cross"] >= lo) & (rec["a_cross"] < hi)
    assert mw.sum() == rec["k"][inw].sum()
    # per record: its pixel is the one of its direction from the box centre
    sel = np.nonzero(inw)[0][:50]
    for r in sel:
        one = O.skymap(P, rec[r:r + 1], 8, lo, hi)
        assert one[O.ang2pix(8, rec["x"][r] - 8.0)] == rec["k"][r]


def test_lcdensity_cells():
    P = O.params(n1d=8, mesh=16, box=16.0)
    rng = np.random.default_rng(4)
    rec = np.zeros(3000, O.RECORD_DTYPE)
    rec["k"] = rng.integers(1, 9, size=3000)
    rec["a_cross"] = rng.uniform(0.02, 1.0, size=3000)
    rec["x"] = rng.uniform(0, 16.0, size=(3000, 3))
    rec["x"][0] = [0.0, 15.999999999, 8.0]
    g = O.lcdensity(P, rec, 32)
    assert g.sum() == rec["k"].sum()
    assert g[0, 31, 16] >= rec["k"][0]
    # brute force: cell of each record by exact comparison with the cell edges
    want = np.zeros((32, 32, 32), np.uint64)
    for r in rec:
        c = [int(np.searchsorted(np.arange(1, 32) * 0.5, x, side="right")) for x in r["x"]]
        want[tuple(c)] += r["k"]
    assert np.array_equal(g, want)
    lo, hi = 0.25, 0.5
    inw = (rec["a_cross"] >= lo) & (rec["a_cross"] < hi)
    assert O.lcdensity(P, rec, 32, lo, hi).sum() == rec["k"][inw].sum()


NS = 8


@pytest.fixture(scope="module")
def angles():
    return sht.pixel_angles(NS)


def test_constant_map(angles):
    c = 3.5
    a = sht.alm(np.full(12 * NS * NS, c), NS, 12, angles)
    assert abs(a[0, 0] - c * math.sqrt(4 * math.pi)) < 1e-12
    assert math.isclose(sht.cl(a)[0], 4 * math.pi * c * c, rel_tol=1e-12)
    # every ring holds 4 i pixels: its phi sum vanishes exactly unless 4 | m;
    # m = 0 and m = 4, 8, ...: the ring quadrature (aliasing in the polar rings)
    nz = [mm for mm in range(1, 13) if mm % 4]
    assert np.abs(a[:, nz]).max() < 1e-12
    assert np.abs(a[1:NS + 1, ::4]).max() < 2e-2 * c  # l <= Nside


def test_dipole_map(angles):
    theta, phi = angles
    a = sht.alm(np.cos(theta), NS, 6, angles)
    assert abs(a[1, 0] / math.sqrt(4 * math.pi / 3) - 1) < 2e-3  # quadrature: 1.5e-3 at Nside 8
    off = np.abs(a).copy()
    off[1, 0] = 0
    assert off.max() < 2e-2


@pytest.mark.parametrize("l,m", [(2, 0), (3, 1), (5, 4), (7, 2)])
def test_single_harmonic(angles, l, m):
    """map = Re Y_lm: a_lm = 1/2 (m > 0) or 1 (m = 0), everything else ~0
    (pixel-centre quadrature, so to ~1e-2 at l < Nside)"""
    from scipy.special import sph_harm_y
    theta, phi = angles
    y = np.real(sph_harm_y(l, m, theta, phi))
    a = sht.alm(y, NS, 10, angles)
    want = 1.0 if m == 0 else 0.5
    assert abs(a[l, m] - want) < 2e-2
    off = np.abs(a).copy()
    off[l, m] = 0
    assert off.max() < 2e-2
    assert abs(sht.alm_one(y, NS, l, m, angles) - a[l, m]) < 1e-13


def test_ylm_routes_agree():
    """the three library routes to Y_lm agree where they overlap"""
    mpmath = pytest.importorskip("mpmath")
    from scipy.special import sph_harm_y
    th = np.array([0.05, 0.7, 1.5707963267948966, 2.9])
    ph = np.array([0.3, 1.1, 4.0, 6.0])
    for l, m in [(3, 0), (40, 0), (40, 13), (500, 250), (599, 3)]:
        a = sht.ylm(l, m, th, ph)
        b = sht._ylm_mpmath(l, m, th, ph)
        c = sph_harm_y(l, m, th, ph)
        assert np.allclose(a, b, rtol=0, atol=1e-11)
        assert np.allclose(c, b, rtol=0, atol=1e-11)
    # past scipy's range: finite, and orthonormal over a fine theta grid
    x, w = np.polynomial.legendre.leggauss(1200)
    t = np.arccos(x)
    y = sht.ylm(767, 383, t, np.zeros_like(t)).real
    assert np.all(np.isfinite(y))
    assert abs(2 * np.pi * np.sum(w * y * y) - 1) < 1e-9


# ---------------------------------------------------------------- P(k)

def test_pk_bins_integer_rounding():
    from oracle import pk
    b, n2 = pk.mode_bins(16)
    r = np.sqrt(n2)
    nz = n2 > 0
    assert np.all((b[nz] - 0.5) ** 2 <= n2[nz]) and np.all(n2 < (b + 0.5) ** 2)
    assert b[0, 0, 0] == 0 and b[1, 0, 0] == 1 and b[1, 1, 0] == 1 and b[1, 1, 1] == 2
    assert np.all(np.abs(b - r) <= 0.5)


@pytest.mark.parametrize("n0", [(3, 0, 0), (2, 2, 1), (0, 5, 4)])
def test_pk_single_mode(n0):
    """delta = A cos(2 pi n0.x / M): all power A^2 L^3 / 2 (modes +-n0) in the
    bin round(|n0|), nothing elsewhere"""
    from oracle import pk
    P = O.params(n1d=8, mesh=16, box=40.0)
    M, A = 16, 0.3
    i = np.arange(M)
    ph = 2 * np.pi * (n0[0] * i[:, None, None] + n0[1] * i[None, :, None] + n0[2] * i[None, None, :]) / M
    delta = A * np.cos(ph)
    k, p, nm = pk.pk_from_delta(P, delta, 7, deconvolve=False)
    tot = p * nm
    b = int(round(math.sqrt(sum(x * x for x in n0))))
    assert math.isclose(tot[b - 1], A * A * P.box ** 3 / 2, rel_tol=1e-12)
    assert np.abs(np.delete(tot, b - 1)).max() < 1e-12 * tot[b - 1]
    assert np.all(nm > 0) and math.isclose(k[0], 2 * np.pi / P.box * np.mean(
        np.sqrt(pk.mode_bins(M)[1][pk.mode_bins(M)[0] == 1])), rel_tol=1e-14)


def test_pk_poisson_sample():
    """uniform random unit-mass particles: the deconvolved power equals the
    CIC shot-noise closed form P_shot C(k) / W(k)^2, C = prod (1 - 2/3 sin^2(pi
    n_i / M)) (the sum over aliases of the CIC window, Jing 2005), so the
    shot-subtracted P(k) is P_shot (C / W^2 - 1) within sample variance"""
    from oracle import pk
    rng = np.random.default_rng(11)
    P = O.params(n1d=32, mesh=32, box=64.0)
    n = 32 ** 3
    u = rng.integers(0, 2 ** 32, size=(3, n), dtype=np.uint64).astype(np.uint32)
    k = np.ones(n, np.uint32)
    kk, pw, nm = pk.power_spectrum(P, u, k, 15)
    shot = P.box ** 3 / n
    M = 32
    s = np.fft.fftfreq(M, 1.0 / M)
    w1 = np.sinc(s / M) ** 2
    c1 = 1 - 2.0 / 3.0 * np.sin(np.pi * s / M) ** 2
    ratio = (c1[:, None, None] * c1[None, :, None] * c1[None, None, :]) / (
        w1[:, None, None] * w1[None, :, None] * w1[None, None, :]) ** 2
    b, _ = pk.mode_bins(M)
    for j in range(1, 16):
        want = shot * (ratio[b == j].mean() - 1)
        sig = shot * ratio[b == j].mean() / math.sqrt(nm[j - 1] / 2)  # Hermitian pairs
        assert abs(pw[j - 1] - want) < 5 * sig, (j, pw[j - 1], want, sig)


def test_pk_of_initial_conditions_is_linear_theory():
    """the ICs' particles at z = 49 follow P_lin(k) D+(a_i)^2 bin by bin.  A
    displaced lattice carries no Poisson shot noise: nothing is subtracted"""
    from oracle import pk
    P = O.params(n1d=32, mesh=64, box=256.0, seed=3)
    st = O.ics(P)
    k, p, nm = pk.power_spectrum(P, st["u"], st["k"], 12, subtract_shot=False)
    D = O.growth(P, 1 / 50)
    for j in range(12):
        want = O.power(P, k[j]) * D * D
        assert abs(p[j] / want - 1) < 5 * math.sqrt(2.0 / nm[j]), (j, p[j], want)



def test_dzs_vs_std_lightcone_within_paper_accuracy():
    """Sec. 3.1.2: the sky-projected lightcone of a DZS run matches the
    standard run's to <= 0.1% (here identical, like the paper's SMALL pair);
    the 3D lightcone and the angular power spectrum too.  16^3, L = 32, FP64
    oracle, full runs from the same ICs."""
    def run(P):
        st = O.initial_state(P)
        recs = []
        for n in range(P.nsteps):
            st, rec = O.step(P, n, st)
            recs.append(rec)
        return st, np.concatenate(recs)
    kw = dict(n1d=16, mesh=32, box=32.0, merge_level=2)
    std_st, std_rec = run(O.params(**kw, dzs_on=0))
    dzs_st, dzs_rec = run(O.params(**kw, dzs_on=1))
    P = O.params(**kw)
    assert dzs_st["u"].shape[1] < 0.6 * std_st["u"].shape[1]  # DZS did de-refine
    assert dzs_rec["k"].sum() == std_rec["k"].sum() == 16 ** 3
    for nside in (4, 16):
        a = O.skymap(P, std_rec, nside).astype(float)
        b = O.skymap(P, dzs_rec, nside).astype(float)
        assert np.abs(a - b).sum() <= 1e-3 * a.sum()
    ga = O.lcdensity(P, std_rec, 16).astype(float)
    gb = O.lcdensity(P, dzs_rec, 16).astype(float)
    assert np.abs(ga - gb).sum() <= 1e-3 * ga.sum()
    ca = sht.cl(sht.alm(O.skymap(P, std_rec, 8).astype(float), 8, 16))
    cb = sht.cl(sht.alm(O.skymap(P, dzs_rec, 8).astype(float), 8, 16))
    assert np.all(np.abs(cb / ca - 1) <= 1e-3)
