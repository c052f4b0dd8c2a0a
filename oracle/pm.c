/*
 * pm.c -- oracle: particle-mesh long-range force.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper's TreePM solves Poisson's equation on an auxiliary uniform mesh in
 * Fourier space and joins it to the tree force with an exponential kernel
 * (Sec. 2.1).  The details are not printed; the reading used is the standard
 * one of the code the paper builds on:
 *   - cloud-in-cell (CIC) assignment to mesh nodes at i * L / M, periodic;
 *     delta = n / nbar - 1 with n the assigned mass in units of m0 and
 *     nbar = N0 / M^3;
 *   - phi_k = -1.5 Om delta_k exp(-k^2 r_s^2) / k^2 / W(k)^2,
 *     W = prod_i sinc^2(pi n_i / M) (assignment and interpolation both
 *     deconvolved), k = 0 -> 0 (nabla^2 phi = 4 pi G rho_bar delta with
 *     4 pi G rho_bar = 1.5 Om for H0 = 1);
 *   - g = -grad phi with the four-point difference
 *     [8 (phi_{+1} - phi_{-1}) - (phi_{+2} - phi_{-2})] / (12 Delta) at the nodes,
 *     interpolated to the particles with the same CIC weights.
 * Mesh index (ix, iy, iz) is stored at (ix M + iy) M + iz.
 */
#include <math.h>
#include <stdlib.h>

#include "oracle.h"

/* node index and weight fraction along one axis: u M / 2^32 = i + f */
static void cic_axis(uint32_t u, int M, int* i0, int* i1, double* f) {
  uint64_t t = (uint64_t)u * (uint64_t)M;
  *i0 = (int)(t >> 32);
  *i1 = (*i0 + 1) % M;
  *f = (double)(t & 0xFFFFFFFFull) * 0x1.0p-32;
}

void dzso_cic_delta(const dzso_params* P, int64_t n, const uint32_t* u,
                    const uint32_t* k, double* delta) {
  int M = P->mesh;
  size_t m3 = (size_t)M * M * M;
  for (size_t c = 0; c < m3; ++c) delta[c] = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    int lo[3], hi[3];
    double f[3];
    for (int ax = 0; ax < 3; ++ax) cic_axis(u[(size_t)ax * n + i], M, &lo[ax], &hi[ax], &f[ax]);
    for (int o = 0; o < 8; ++o) {
      int ox = (o >> 2) & 1, oy = (o >> 1) & 1, oz = o & 1;
      double w = (ox ? f[0] : 1.0 - f[0]) * (oy ? f[1] : 1.0 - f[1]) * (oz ? f[2] : 1.0 - f[2]);
      size_t c = ((size_t)(ox ? hi[0] : lo[0]) * M + (oy ? hi[1] : lo[1])) * M + (oz ? hi[2] : lo[2]);
      delta[c] += (double)k[i] * w;
    }
  }
  double n0 = (double)P->n1d * P->n1d * P->n1d;
  double nbar = n0 / (double)m3;
  for (size_t c = 0; c < m3; ++c) delta[c] = delta[c] / nbar - 1.0;
}

static int wavenumber_index(int m, int n) { return (m <= n / 2) ? m : m - n; }

static double sinc(double x) { return x == 0.0 ? 1.0 : sin(x) / x; }

void dzso_pm_potential(const dzso_params* P, const double* delta, double* phi) {
  int M = P->mesh;
  size_t m3 = (size_t)M * M * M;
  double L = P->box;
  double kf = 2.0 * M_PI / L;
  double rs = P->rs_cells * L / M;
  double* x = (double*)malloc(sizeof(double) * 2 * m3);
  for (size_t c = 0; c < m3; ++c) {
    x[2 * c] = delta[c];
    x[2 * c + 1] = 0.0;
  }
  dzso_fft3(M, M, M, x, -1);
  for (int a = 0; a < M; ++a)
    for (int b = 0; b < M; ++b)
      for (int c = 0; c < M; ++c) {
        size_t idx = ((size_t)a * M + b) * M + c;
        int na = wavenumber_index(a, M), nb = wavenumber_index(b, M), nc = wavenumber_index(c, M);
        double k2 = kf * kf * ((double)na * na + (double)nb * nb + (double)nc * nc);
        double g = 0.0;
        if (k2 > 0.0) {
          double w = sinc(M_PI * na / M) * sinc(M_PI * nb / M) * sinc(M_PI * nc / M);
          w = w * w; /* W_CIC = prod sinc^2 */
          g = -1.5 * P->omega_m * exp(-k2 * rs * rs) / k2 / (w * w);
        }
        x[2 * idx] *= g;
        x[2 * idx + 1] *= g;
      }
  dzso_fft3(M, M, M, x, +1);
  for (size_t c = 0; c < m3; ++c) phi[c] = x[2 * c] / (double)m3;
  free(x);
}

static double phi_at(const double* phi, int M, int a, int b, int c) {
  a = ((a % M) + M) % M;
  b = ((b % M) + M) % M;
  c = ((c % M) + M) % M;
  return phi[((size_t)a * M + b) * M + c];
}

/* -dphi/dx_ax at node (a, b, c), four-point stencil */
static double neg_grad(const double* phi, int M, double dx, int ax, int a, int b, int c) {
  int e[3] = {0, 0, 0};
  e[ax] = 1;
  double p1 = phi_at(phi, M, a + e[0], b + e[1], c + e[2]);
  double m1 = phi_at(phi, M, a - e[0], b - e[1], c - e[2]);
  double p2 = phi_at(phi, M, a + 2 * e[0], b + 2 * e[1], c + 2 * e[2]);
  double m2 = phi_at(phi, M, a - 2 * e[0], b - 2 * e[1], c - 2 * e[2]);
  return -(8.0 * (p1 - m1) - (p2 - m2)) / (12.0 * dx);
}

static void pm_one(const dzso_params* P, const double* phi, int64_t n,
                   const uint32_t* u, double* g, int64_t i) {
  int M = P->mesh;
  double dx = P->box / M;
  int lo[3], hi[3];
  double f[3];
  for (int ax = 0; ax < 3; ++ax) cic_axis(u[(size_t)ax * n + i], M, &lo[ax], &hi[ax], &f[ax]);
  double acc[3] = {0.0, 0.0, 0.0};
  for (int o = 0; o < 8; ++o) {
    int ox = (o >> 2) & 1, oy = (o >> 1) & 1, oz = o & 1;
    double w = (ox ? f[0] : 1.0 - f[0]) * (oy ? f[1] : 1.0 - f[1]) * (oz ? f[2] : 1.0 - f[2]);
    int a = ox ? hi[0] : lo[0], b = oy ? hi[1] : lo[1], c = oz ? hi[2] : lo[2];
    for (int ax = 0; ax < 3; ++ax) acc[ax] += w * neg_grad(phi, M, dx, ax, a, b, c);
  }
  for (int ax = 0; ax < 3; ++ax) g[(size_t)ax * n + i] = acc[ax];
}

void dzso_pm_accel(const dzso_params* P, const double* phi, int64_t n,
                   const uint32_t* u, double* g, const int64_t* sample,
                   int64_t nsample) {
  if (nsample > 0) {
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < nsample; ++s) pm_one(P, phi, n, u, g, sample[s]);
  } else {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) pm_one(P, phi, n, u, g, i);
  }
}
