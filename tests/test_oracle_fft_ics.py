"""Pins of the oracle FFT (oracle/fft.c) and initial conditions (oracle/ics.c).

FFT: naive DFT on small sizes (radix 2 and 3), numpy.fft, round trip.
ICs: the published SplitMix64 stream, Gaussian moments, the measured power
spectrum of the displacement divergence vs the input P(k), zero mean
displacement, and the Zel'dovich momentum / displacement relation."""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def naive_dft(x, sign):
    n = len(x)
    j = np.arange(n)
    return np.array([(x * np.exp(sign * 2j * np.pi * j * kk / n)).sum() for kk in range(n)])


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 8, 9, 12, 18, 24, 48, 7])
def test_fft1_naive(n):
    rng = np.random.default_rng(n)
    x = rng.normal(size=n) + 1j * rng.normal(size=n)
    for sign in (-1, 1):
        assert np.allclose(O.fft1(x, sign), naive_dft(x, sign), rtol=0, atol=1e-13 * max(1, n))


@pytest.mark.parametrize("shape", [(8, 8, 8), (12, 12, 12), (4, 6, 3)])
def test_fft3_numpy_and_roundtrip(shape):
    rng = np.random.default_rng(7)
    x = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    f = O.fft3(x, -1)
    assert np.allclose(f, np.fft.fftn(x), rtol=0, atol=1e-12)
    b = O.fft3(f, +1) / x.size
    assert np.allclose(b, x, rtol=0, atol=1e-14)


def test_splitmix64_published_stream():
    lines = open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt")).read().splitlines()
    want = [int(v) for v in lines if v.strip() and not v.startswith("#")]
    assert len(want) == 3
    assert [O.splitmix64_at(1234567, c) for c in range(3)] == want


def test_white_noise_moments():
    w = O.white_noise(42, 32)
    assert abs(w.mean()) < 4 / math.sqrt(w.size)
    assert abs(w.var() - 1) < 5 * math.sqrt(2 / w.size)
    # 4th moment of a Gaussian is 3
    assert abs((w ** 4).mean() - 3) < 0.15


def _ics(n1d=32, box=64.0, seed=1):
    P = O.params(n1d=n1d, box=box, mesh=2 * n1d, seed=seed)
    st = O.ics(P)
    return P, st


def _psi(P, st):
    """Displacement field (Mpc/h) on the lattice, [3, n1, n1, n1]."""
    from oracle_util import lattice_positions
    n1 = P.n1d
    q = lattice_positions(n1, P.box)
    du = (st["u"].astype(np.int64) - q.astype(np.int64))
    du = (du + (1 << 31)) % (1 << 32) - (1 << 31)
    return (du * (P.box / 2.0 ** 32)).reshape(3, n1, n1, n1)


def test_ics_mean_displacement_and_momentum_relation():
    P, st = _ics()
    psi_d = _psi(P, st)  # = D+(a_i) psi
    # k = 0 mode removed: mean displacement ~ 0 (up to lattice rounding)
    assert np.all(np.abs(psi_d.mean(axis=(1, 2, 3))) < 1e-6)
    ai = 1 / 50
    fac = ai ** 2 * O.hubble_e(P, ai) * O.growth_rate(P, ai)  # p = a^2 E f (D psi)
    p = st["p"].reshape(3, P.n1d, P.n1d, P.n1d)
    lat = P.box / 2.0 ** 32
    assert np.allclose(p, fac * psi_d, rtol=0, atol=fac * lat)
    assert np.array_equal(st["k"], np.ones(P.n1d ** 3, np.uint32))
    assert np.array_equal(st["id"], np.arange(P.n1d ** 3, dtype=np.uint32))


def test_ics_power_spectrum_matches_input():
    """delta = -div(psi); its binned |delta_k|^2 L^3 / n^6 divided by D+(a_i)^2
    must match P(k) within sample variance (chi^2 per bin)."""
    P, st = _ics(n1d=32, box=256.0, seed=3)
    n1 = P.n1d
    psi = _psi(P, st)
    kf = 2 * np.pi * np.fft.fftfreq(n1, d=1.0 / n1) / P.box
    kx, ky, kz = np.meshgrid(kf, kf, kf, indexing="ij")
    dk = np.zeros((n1, n1, n1), complex)
    for ax, kk in enumerate((kx, ky, kz)):
        # drop each axis' Nyquist plane, as the ICs do
        pk = np.fft.fftn(psi[ax])
        nyq = np.zeros_like(kk, bool)
        idx = [slice(None)] * 3
        idx[ax] = n1 // 2
        nyq[tuple(idx)] = True
        dk += np.where(nyq, 0, -1j * kk * pk)
    kmag = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    D = O.growth(P, 1 / 50)
    pow_meas = np.abs(dk) ** 2 * P.box ** 3 / n1 ** 6 / D ** 2
    kfund = 2 * np.pi / P.box
    bins = np.arange(0.5, n1 // 2 - 1, 1.0) * kfund
    chi2, nb = 0.0, 0
    for lo, hi in zip(bins[:-1], bins[1:]):
        sel = (kmag >= lo) & (kmag < hi)
        nm = sel.sum()
        if nm < 20:
            continue
        kmean = kmag[sel].mean()
        want = np.mean([O.power(P, x) for x in np.quantile(kmag[sel], [0.25, 0.5, 0.75])])
        got = pow_meas[sel].mean()
        sig = want * math.sqrt(2.0 / nm)  # modes counted twice (Hermitian pairs)
        chi2 += ((got - want) / sig) ** 2
        nb += 1
        assert abs(got / want - 1) < 6 * math.sqrt(2.0 / nm) + 0.05, (kmean, got, want)
    assert nb >= 8
    assert chi2 / nb < 3.0
