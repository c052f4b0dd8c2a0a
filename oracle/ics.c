/*
 * ics.c -- oracle: Zel'dovich initial conditions from a seeded Gaussian field.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper starts from initial conditions evolved with linear theory to
 * z >~ 50 (Fig. 1 caption) and does not print the recipe; the reading used
 * here is the textbook one:
 *   white noise w on the n^3 particle lattice, drawn with SplitMix64
 *   (Steele, Lea & Flood 2014) as a counter-based generator and Box-Muller;
 *   delta_k = W_k sqrt(n^3 P(k) / L^3)   (forward FFT unnormalised);
 *   psi_k   = i k delta_k / k^2, k = 0 and each axis' Nyquist plane -> 0;
 *   x = q + D+(a_i) psi,   p = a^2 dx/dt = a_i^3 E(a_i) dD+/da psi.
 * Lattice q = (i, j, l) * L / n at cell corners; id = (i n + j) n + l.
 */
#include <math.h>
#include <stdlib.h>

#include "oracle.h"

#define GOLDEN_GAMMA 0x9E3779B97F4A7C15ull

static uint64_t splitmix64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* the c-th output (c >= 0) of a SplitMix64 stream whose state starts at seed */
uint64_t dzso_splitmix64_at(uint64_t seed, uint64_t c) {
  return splitmix64_mix(seed + (c + 1) * GOLDEN_GAMMA);
}

/* unit-variance Gaussian for lattice index idx: outputs 2 idx and 2 idx + 1
 * give u1 in (0, 1] and u2 in [0, 1); w = sqrt(-2 ln u1) cos(2 pi u2) */
void dzso_white_noise(uint64_t seed, int n1d, double* w) {
  int64_t n = (int64_t)n1d * n1d * n1d;
  for (int64_t idx = 0; idx < n; ++idx) {
    uint64_t r0 = dzso_splitmix64_at(seed, 2 * (uint64_t)idx);
    uint64_t r1 = dzso_splitmix64_at(seed, 2 * (uint64_t)idx + 1);
    double u1 = ((double)(r0 >> 11) + 1.0) * 0x1.0p-53;
    double u2 = (double)(r1 >> 11) * 0x1.0p-53;
    w[idx] = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
  }
}

static int wavenumber_index(int m, int n) { return (m <= n / 2) ? m : m - n; }

void dzso_ics(const dzso_params* P, uint32_t* u, double* p, uint32_t* k,
              uint32_t* id, uint8_t* fl) {
  int n1 = P->n1d;
  int64_t n = (int64_t)n1 * n1 * n1;
  double L = P->box;
  double ai = 1.0 / (1.0 + P->z_init);
  double amp = dzso_power_amplitude(P);
  double dplus = dzso_growth(P, ai);
  double fgrow = dzso_growth_rate(P, ai);
  double ei = dzso_hubble_e(P, ai);
  /* p = a^3 E dD/da psi = a^2 E f D psi */
  double pfac = ai * ai * ei * fgrow * dplus;
  double kf = 2.0 * M_PI / L;

  double* w = (double*)malloc(sizeof(double) * (size_t)n);
  dzso_white_noise(P->seed, n1, w);
  double* dk = (double*)malloc(sizeof(double) * 2 * (size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    dk[2 * i] = w[i];
    dk[2 * i + 1] = 0.0;
  }
  free(w);
  dzso_fft3(n1, n1, n1, dk, -1);
  /* delta_k */
  double norm = (double)n / (L * L * L);
  for (int a = 0; a < n1; ++a)
    for (int b = 0; b < n1; ++b)
      for (int c = 0; c < n1; ++c) {
        size_t idx = ((size_t)a * n1 + b) * n1 + c;
        int na = wavenumber_index(a, n1), nb = wavenumber_index(b, n1), nc = wavenumber_index(c, n1);
        double kk = kf * sqrt((double)na * na + (double)nb * nb + (double)nc * nc);
        double s = (kk > 0.0) ? sqrt(norm * amp * dzso_power_shape(P, kk)) : 0.0;
        dk[2 * idx] *= s;
        dk[2 * idx + 1] *= s;
      }

  double* psi = (double*)malloc(sizeof(double) * 2 * (size_t)n);
  for (int ax = 0; ax < 3; ++ax) {
    for (int a = 0; a < n1; ++a)
      for (int b = 0; b < n1; ++b)
        for (int c = 0; c < n1; ++c) {
          size_t idx = ((size_t)a * n1 + b) * n1 + c;
          int nv[3] = {wavenumber_index(a, n1), wavenumber_index(b, n1), wavenumber_index(c, n1)};
          int mv[3] = {a, b, c};
          double k2 = kf * kf * ((double)nv[0] * nv[0] + (double)nv[1] * nv[1] + (double)nv[2] * nv[2]);
          double re = 0.0, im = 0.0;
          int nyq = (n1 % 2 == 0) && (mv[ax] == n1 / 2);
          if (k2 > 0.0 && !nyq) {
            double kc = kf * nv[ax] / k2;
            /* i kc (x + i y) = -kc y + i kc x */
            re = -kc * dk[2 * idx + 1];
            im = kc * dk[2 * idx];
          }
          psi[2 * idx] = re;
          psi[2 * idx + 1] = im;
        }
    dzso_fft3(n1, n1, n1, psi, +1);
    double lat = 4294967296.0 / L;
    for (int a = 0; a < n1; ++a)
      for (int b = 0; b < n1; ++b)
        for (int c = 0; c < n1; ++c) {
          size_t idx = ((size_t)a * n1 + b) * n1 + c;
          int mv[3] = {a, b, c};
          double ps = psi[2 * idx] / (double)n;
          uint64_t q = ((uint64_t)mv[ax] << 32) / (uint64_t)n1;
          int64_t du = llrint(dplus * ps * lat);
          u[(size_t)ax * n + idx] = (uint32_t)(q + (uint64_t)du);
          p[(size_t)ax * n + idx] = pfac * ps;
        }
  }
  free(psi);
  free(dk);
  for (int64_t i = 0; i < n; ++i) {
    k[i] = 1;
    id[i] = (uint32_t)i;
    fl[i] = 0;
  }
}
