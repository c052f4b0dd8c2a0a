"""Oracle: 3D matter power spectrum of the particle set (the final P(k)
compared between DZS and standard runs; the paper itself prefers lightcone
observables, Sec. 3.1, and P(k) is kept as a time-slice check).

TEST INFRASTRUCTURE ONLY (see oracle.h).

Plain definition on the oracle's own CIC mesh (mass-weighted,
delta = n / nbar - 1 on the nodes iL/M):
    delta_k = sum_x delta(x) e^{-i k.x}              (numpy.fft.fftn, all modes)
    P_mode  = |delta_k|^2 L^3 / M^6 / W(k)^2 - P_shot
    W(k)    = prod_i sinc^2(pi n_i / M)              (CIC assignment window)
    P_shot  = L^3 sum k_j^2 / (sum k_j)^2             (particles of mass k_j m0;
                                                       optional: meant for Poisson-like sets)
Bins: mode n (integer vector, |n| = |k| / k_f, k_f = 2 pi / L) belongs to bin
b = round(|n|), i.e. (b - 1/2)^2 <= |n|^2 < (b + 1/2)^2 tested on integers;
b = 1 .. nbins.  Per bin: the number of modes, the mean |k| and the mean
P_mode.
"""
from __future__ import annotations

import numpy as np

from . import cic_delta


def mode_bins(M):
    """integer bin of every mode of an M^3 complex grid (fftn order)"""
    s = np.fft.fftfreq(M, 1.0 / M).astype(np.int64)
    n2 = s[:, None, None] ** 2 + s[None, :, None] ** 2 + s[None, None, :] ** 2
    r = np.floor(np.sqrt(4.0 * n2)).astype(np.int64)  # floor sqrt(4 n^2), fixed up exactly
    r = np.where(r * r > 4 * n2, r - 1, r)
    r = np.where((r + 1) ** 2 <= 4 * n2, r + 1, r)
    return (r + 1) // 2, n2


def pk_from_delta(P, delta, nbins, shot=0.0, deconvolve=True):
    M = delta.shape[0]
    L = P.box
    dk = np.fft.fftn(delta)
    pw = np.abs(dk) ** 2 * L ** 3 / float(M) ** 6
    if deconvolve:
        s = np.fft.fftfreq(M, 1.0 / M)
        w1 = np.sinc(s / M) ** 2  # np.sinc(x) = sin(pi x) / (pi x)
        W = w1[:, None, None] * w1[None, :, None] * w1[None, None, :]
        pw = pw / (W * W)
    pw = pw - shot
    b, n2 = mode_bins(M)
    kmag = 2.0 * np.pi / L * np.sqrt(n2)
    out_k = np.zeros(nbins)
    out_p = np.zeros(nbins)
    out_n = np.zeros(nbins)
    for j in range(1, nbins + 1):
        sel = b == j
        out_n[j - 1] = sel.sum()
        out_k[j - 1] = kmag[sel].mean()
        out_p[j - 1] = pw[sel].mean()
    return out_k, out_p, out_n


def power_spectrum(P, u, k, nbins, subtract_shot=True):
    """(k, P(k), modes) of the particles u [3, n] (uint32 lattice), masses k"""
    k = np.asarray(k)
    delta = cic_delta(P, u, k).reshape(P.mesh, P.mesh, P.mesh)
    kk = k.astype(np.float64)
    shot = P.box ** 3 * float((kk * kk).sum()) / float(kk.sum()) ** 2 if subtract_shot else 0.0
    return pk_from_delta(P, delta, nbins, shot=shot)
