"""Oracle: spherical-harmonic coefficients and angular power spectrum of a
RING-ordered equal-area sky map (the paper's Fig. 4 bottom row compares the
angular power spectra of the DZS and standard lightcone maps).

TEST INFRASTRUCTURE ONLY (see oracle.h).

Plain definition, no fast transform: with pixel centres (theta_p, phi_p) from
the oracle's pixelisation and the pixel solid angle Omega = 4 pi / N_pix,

    a_lm = Omega * sum_p map_p * conj(Y_lm(theta_p, phi_p)),   0 <= m <= l,
    C_l  = (|a_l0|^2 + 2 sum_{m>=1} |a_lm|^2) / (2 l + 1),

Y_lm the orthonormal spherical harmonics with the Condon-Shortley phase,
taken from library routines: Y_l0 = sqrt((2l+1)/(4 pi)) P_l(cos theta) with
scipy.special.eval_legendre; m > 0 from scipy.special.sph_harm_y, which
returns NaN above l ~ 600, where mpmath.spherharm (arbitrary precision,
evaluated once per distinct theta) is used instead.  For a real map a_l,-m =
(-1)^m conj(a_lm), so m >= 0 carries all of it.
"""
from __future__ import annotations

import numpy as np
from scipy.special import eval_legendre, sph_harm_y

from . import pix2zphi


def pixel_angles(nside):
    """(theta, phi) of every pixel centre, RING order"""
    z, phi = pix2zphi(nside, np.arange(12 * nside * nside))
    return np.arccos(np.clip(z, -1.0, 1.0)), phi


def _ylm_mpmath(l, mm, theta, phi):
    try:
        import mpmath
    except ImportError as e:  # pragma: no cover - depends on the host
        raise RuntimeError("Y_lm above l ~ 600 needs mpmath") from e
    mpmath.mp.dps = 30
    ut, inv = np.unique(theta, return_inverse=True)
    lam = np.array([float(mpmath.re(mpmath.spherharm(l, mm, t, 0))) for t in ut])
    return lam[inv] * np.exp(1j * mm * phi)


def ylm(l, mm, theta, phi):
    """Y_{l mm}(theta, phi) for one degree and order, 0 <= mm <= l"""
    if mm == 0:
        return np.sqrt((2 * l + 1) / (4 * np.pi)) * eval_legendre(l, np.cos(theta)) + 0j
    y = sph_harm_y(l, mm, theta, phi)
    if np.isnan(y).any():
        y = _ylm_mpmath(l, mm, theta, phi)
    return y


def alm(m, nside, lmax, angles=None):
    """a_lm as a complex array [lmax + 1, lmax + 1] indexed [l, m] (0 for m > l)"""
    m = np.asarray(m, np.float64)
    theta, phi = angles if angles is not None else pixel_angles(nside)
    omega = 4.0 * np.pi / m.size
    out = np.zeros((lmax + 1, lmax + 1), np.complex128)
    for mm in range(lmax + 1):
        for l in range(mm, lmax + 1):
            out[l, mm] = omega * (np.conj(ylm(l, mm, theta, phi)) @ m)
    return out


def alm_one(m, nside, l, mm, angles=None):
    """a single coefficient a_{l mm}"""
    m = np.asarray(m, np.float64)
    theta, phi = angles if angles is not None else pixel_angles(nside)
    return 4.0 * np.pi / m.size * np.sum(np.conj(ylm(l, mm, theta, phi)) * m)


def cl(a):
    """C_l from a_lm [l, m]"""
    lmax = a.shape[0] - 1
    p = np.abs(a) ** 2
    return (p[:, 0] + 2.0 * p[:, 1:].sum(axis=1)) / (2.0 * np.arange(lmax + 1) + 1.0)
