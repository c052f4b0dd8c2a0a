/*
 * fft.c -- oracle: plain mixed-radix complex FFT (recursive Cooley-Tukey,
 * decimation in time, any factorisation; prime lengths fall back to the
 * direct sum).  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Convention: X_k = sum_n x_n exp(sign * 2 pi i n k / N), unnormalised;
 * sign = -1 forward, +1 backward.  The PM solver of the paper works in Fourier
 * space (Sec. 2.1); this is the textbook transform it needs, kept simple so a
 * reader can check it by eye.  Data are interleaved (re, im) doubles.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

static int smallest_factor(int n) {
  for (int r = 2; r * r <= n; ++r)
    if (n % r == 0) return r;
  return n;
}

/* out[k] = sum_j in[j * stride] w^(j k), length n, w = exp(sign 2 pi i / n) */
static void fft_rec(int n, const double* in, int stride, double* out, int sign) {
  if (n == 1) {
    out[0] = in[0];
    out[1] = in[1];
    return;
  }
  int r = smallest_factor(n);
  int m = n / r;
  /* r sub-transforms of length m over the residues j mod r */
  double* sub = (double*)malloc(sizeof(double) * 2 * (size_t)n);
  for (int j = 0; j < r; ++j) fft_rec(m, in + 2 * (size_t)j * stride, stride * r, sub + 2 * (size_t)j * m, sign);
  /* combine: X[q + m s] = sum_j w^(j (q + m s)) Sub_j[q] */
  for (int q = 0; q < m; ++q) {
    for (int s = 0; s < r; ++s) {
      int kk = q + m * s;
      double re = 0.0, im = 0.0;
      for (int j = 0; j < r; ++j) {
        long t = ((long)j * kk) % n; /* reduce the angle exactly */
        double ang = sign * 2.0 * M_PI * (double)t / (double)n;
        double c = cos(ang), sn = sin(ang);
        double xr = sub[2 * ((size_t)j * m + q)], xi = sub[2 * ((size_t)j * m + q) + 1];
        re += xr * c - xi * sn;
        im += xr * sn + xi * c;
      }
      out[2 * (size_t)kk] = re;
      out[2 * (size_t)kk + 1] = im;
    }
  }
  free(sub);
}

void dzso_fft1(int n, double* x, int sign) {
  double* out = (double*)malloc(sizeof(double) * 2 * (size_t)n);
  fft_rec(n, x, 1, out, sign);
  memcpy(x, out, sizeof(double) * 2 * (size_t)n);
  free(out);
}

/* 3D transform of a C-ordered [n0][n1][n2] complex array, one axis at a time */
void dzso_fft3(int n0, int n1, int n2, double* x, int sign) {
  int dims[3] = {n0, n1, n2};
  size_t strides[3] = {(size_t)n1 * n2, (size_t)n2, 1};
  for (int ax = 0; ax < 3; ++ax) {
    int n = dims[ax];
    int oa = (ax + 1) % 3, ob = (ax + 2) % 3;
#pragma omp parallel for collapse(2) schedule(static)
    for (int ia = 0; ia < dims[oa]; ++ia) {
      for (int ib = 0; ib < dims[ob]; ++ib) {
        double* line = (double*)malloc(sizeof(double) * 2 * (size_t)n);
        size_t base = (size_t)ia * strides[oa] + (size_t)ib * strides[ob];
        for (int t = 0; t < n; ++t) {
          line[2 * t] = x[2 * (base + (size_t)t * strides[ax])];
          line[2 * t + 1] = x[2 * (base + (size_t)t * strides[ax]) + 1];
        }
        dzso_fft1(n, line, sign);
        for (int t = 0; t < n; ++t) {
          x[2 * (base + (size_t)t * strides[ax])] = line[2 * t];
          x[2 * (base + (size_t)t * strides[ax]) + 1] = line[2 * t + 1];
        }
        free(line);
      }
    }
  }
}
