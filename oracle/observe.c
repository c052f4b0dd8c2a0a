/*
 * observe.c -- oracle: lightcone observables.  TEST INFRASTRUCTURE ONLY (see
 * oracle.h).
 *
 * Paper Sec. 3.1.2 (sky-projected lightcone): the mass of the lightcone
 * particles is projected on an equal-area sky pixelisation (HEALPix, Górski et
 * al. 2005, the paper's NSIDE = 256 / 1024 maps) and the maps and their
 * angular power spectra of the DZS and standard runs are compared.
 *
 * Pixelisation: the RING ordering of the Górski et al. (2005) scheme, written
 * here from its geometry.  12 Nside^2 pixels of equal area on 4 Nside - 1
 * iso-latitude rings.  Polar caps |z| > 2/3: ring i (1..Nside-1 from the
 * pole, plus ring Nside) holds 4 i pixels centred at z = +-(1 - i^2 / (3
 * Nside^2)), phi = (j - 1/2) pi / (2 i).  Equatorial belt |z| <= 2/3: rings
 * Nside..3 Nside hold 4 Nside pixels at z = 4/3 - 2 i / (3 Nside), phi =
 * (j - f) pi / (2 Nside) with f = 1 on rings where i + Nside is odd, else
 * 1/2.  Pixel boundaries in the belt are the lines Nside (1/2 + t) -+ (3/4)
 * Nside z = integer (t = phi / (pi/2)); in the caps, the lines t' sqrt(3 (1 -
 * |z|)) Nside = integer and (1 - t') sqrt(3 (1 - |z|)) Nside = integer
 * (t' = t - floor(t)).
 *
 * 3D lightcone density (Sec. 3.1.3, Fig. 5: the particle lightcone written
 * on the fly in a thin shell at R_lc): the mass k of each record in the a*
 * window is added to the cell floor(x* / L * M) of an M^3 mesh (nearest grid
 * point, cell [i][j][l] at index (i M + j) M + l).
 *
 * Sky map reading: a lightcone record (Sec. 1 footnote; crossing position x*)
 * is seen in the direction x* - x_obs (x* lies in [0, L), the observer at
 * L/2, so that difference is the minimum image); its mass k is added to the
 * pixel of that direction when a_lo <= a* < a_hi; a record at the observer
 * itself is put in the direction +z.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

static int64_t floor_div(int64_t a, int64_t b) {
  int64_t q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}

static int64_t pos_mod(int64_t a, int64_t b) {
  int64_t r = a % b;
  return r < 0 ? r + b : r;
}

int64_t dzso_ang2pix_ring(int64_t nside, double x, double y, double z) {
  const double r = sqrt(x * x + y * y + z * z);
  const double cz = r > 0.0 ? z / r : 1.0;
  const double za = fabs(cz);
  double phi = (x == 0.0 && y == 0.0) ? 0.0 : atan2(y, x);
  if (phi < 0.0) phi += 2.0 * M_PI;
  double t = phi / (0.5 * M_PI); /* in [0, 4] */
  if (t >= 4.0) t -= 4.0;
  const int64_t npix = 12 * nside * nside;
  if (za <= 2.0 / 3.0) {
    const double a = (double)nside * (0.5 + t), b = (double)nside * 0.75 * cz;
    const int64_t jp = (int64_t)floor(a - b); /* ascending edge line below */
    const int64_t jm = (int64_t)floor(a + b); /* descending edge line below */
    const int64_t ir = nside + 1 + jp - jm;   /* belt ring, 1 .. 2 Nside + 1 */
    const int64_t shift = 1 - (ir & 1);       /* 1 on rings with a pixel centred at phi = 0 */
    const int64_t ip = pos_mod(floor_div(jp + jm - nside + shift, 2), 4 * nside);
    return 2 * nside * (nside - 1) + (ir - 1) * 4 * nside + ip;
  }
  const double tp = t - floor(t);
  const double w = (double)nside * sqrt(3.0 * (1.0 - za));
  const int64_t jp = (int64_t)floor(tp * w), jm = (int64_t)floor((1.0 - tp) * w);
  const int64_t ir = jp + jm + 1; /* ring counted from the nearer pole, 1 .. Nside */
  const int64_t ip = pos_mod((int64_t)floor(t * (double)ir), 4 * ir);
  if (cz > 0.0) return 2 * ir * (ir - 1) + ip;
  return npix - 2 * ir * (ir + 1) + ip;
}

/* largest r with r * r <= v */
static int64_t isqrt64(int64_t v) {
  int64_t r = (int64_t)sqrt((double)v);
  while (r * r > v) --r;
  while ((r + 1) * (r + 1) <= v) ++r;
  return r;
}

void dzso_pix2ring(int64_t nside, int64_t pix, int64_t* ring, int64_t* j, double* z, double* phi) {
  const int64_t npix = 12 * nside * nside, ncap = 2 * nside * (nside - 1);
  int64_t i, jj;
  double zz, ph;
  if (pix < ncap) {
    /* north cap: ring i starts at 2 i (i - 1) */
    i = (1 + isqrt64(1 + 2 * pix)) / 2;
    jj = pix - 2 * i * (i - 1) + 1;
    zz = 1.0 - (double)(i * i) / (3.0 * (double)(nside * nside));
    ph = ((double)jj - 0.5) * M_PI / (2.0 * (double)i);
  } else if (pix < npix - ncap) {
    const int64_t q = pix - ncap;
    i = q / (4 * nside) + nside;
    jj = q % (4 * nside) + 1;
    const double f = ((i + nside) & 1) ? 1.0 : 0.5;
    zz = (double)(2 * nside - i) * 2.0 / (3.0 * (double)nside);
    ph = ((double)jj - f) * M_PI / (2.0 * (double)nside);
  } else {
    /* south cap, ring s from the south pole starts at npix - 2 s (s + 1) */
    const int64_t q = npix - pix;
    const int64_t s = (1 + isqrt64(2 * q - 1)) / 2;
    jj = 4 * s + 1 - (q - 2 * s * (s - 1));
    i = 4 * nside - s;
    zz = -1.0 + (double)(s * s) / (3.0 * (double)(nside * nside));
    ph = ((double)jj - 0.5) * M_PI / (2.0 * (double)s);
  }
  if (ring) *ring = i;
  if (j) *j = jj;
  if (z) *z = zz;
  if (phi) *phi = ph;
}

void dzso_pix2vec_ring(int64_t nside, int64_t pix, double v[3]) {
  double z, phi;
  dzso_pix2ring(nside, pix, NULL, NULL, &z, &phi);
  const double s = sqrt((1.0 - z) * (1.0 + z));
  v[0] = s * cos(phi);
  v[1] = s * sin(phi);
  v[2] = z;
}

void dzso_skymap(const dzso_params* P, int64_t nrec, const dzso_record* rec, int64_t nside, double a_lo,
                 double a_hi, uint64_t* map) {
  const double half = 0.5 * P->box;
  for (int64_t r = 0; r < nrec; ++r) {
    if (!(rec[r].a_cross >= a_lo && rec[r].a_cross < a_hi)) continue;
    int64_t pix = dzso_ang2pix_ring(nside, rec[r].x[0] - half, rec[r].x[1] - half, rec[r].x[2] - half);
    map[pix] += rec[r].k;
  }
}

void dzso_ang2pix_ring_many(int64_t nside, int64_t n, const double* v, int64_t* pix) {
  for (int64_t i = 0; i < n; ++i) pix[i] = dzso_ang2pix_ring(nside, v[i], v[(size_t)n + i], v[2 * (size_t)n + i]);
}

void dzso_pix2vec_ring_many(int64_t nside, int64_t n, const int64_t* pix, double* v) {
  for (int64_t i = 0; i < n; ++i) {
    double w[3];
    dzso_pix2vec_ring(nside, pix[i], w);
    for (int ax = 0; ax < 3; ++ax) v[(size_t)ax * n + i] = w[ax];
  }
}

void dzso_pix2zphi_ring_many(int64_t nside, int64_t n, const int64_t* pix, double* z, double* phi) {
  for (int64_t i = 0; i < n; ++i) dzso_pix2ring(nside, pix[i], NULL, NULL, &z[i], &phi[i]);
}

void dzso_lcdensity(const dzso_params* P, int64_t nrec, const dzso_record* rec, int64_t mesh, double a_lo,
                    double a_hi, uint64_t* grid) {
  for (int64_t r = 0; r < nrec; ++r) {
    if (!(rec[r].a_cross >= a_lo && rec[r].a_cross < a_hi)) continue;
    int64_t c[3];
    for (int ax = 0; ax < 3; ++ax) {
      c[ax] = (int64_t)floor(rec[r].x[ax] / P->box * (double)mesh);
      if (c[ax] < 0) c[ax] = 0;
      if (c[ax] >= mesh) c[ax] = mesh - 1;
    }
    grid[(c[0] * mesh + c[1]) * mesh + c[2]] += rec[r].k;
  }
}
