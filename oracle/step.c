/*
 * step.c -- oracle: kick/drift, lightcone crossing, the full KDK step and the
 * conservation diagnostics.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Step order (paper Sec. 2.2: DZS on global steps, tree rebuilt and forces of
 * new particles recomputed after a merge):
 *   1. opening kick  p += g K(a_n, a_n+1/2)
 *   2. drift         u += rint(p D(a_n, a_n+1) 2^32 / L)   (uint32 wrap)
 *   3. crossing      not yet crossed, d_n < R_lc(a_n) and d_n+1 >= R_lc(a_n+1)
 *                    (Sec. 1 footnote, Sec. 3.1.3: particles are written to
 *                    the lightcone when they meet its boundary); the record
 *                    holds (a*, x*) linearly interpolated to s = d - R = 0
 *   4. Morton sort   (stable)
 *   5. DZS merge     against R_lc(a_n+1)
 *   6. forces        g = PM + tree on the new particle set
 *   7. closing kick  p += g K(a_n+1/2, a_n+1)
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

typedef struct {
  double a0, a1, drift, kick1, kick2, rlc0, rlc1;
  uint64_t rlat0, rlat1;
} step_tab;

static double rlc_of(const dzso_params* P, double a, double chi0) {
  double rmax = sqrt(3.0) * P->box / 2.0;
  double chi = dzso_chi(P, a);
  if (P->rlc_mode == DZSO_RLC_SWEEP) return rmax * chi / chi0;
  return chi < rmax ? chi : rmax;
}

/* the entries of dzso_tables needed by one step, same formulas */
static step_tab step_tables(const dzso_params* P, int step) {
  step_tab t;
  int ns = P->nsteps;
  double lnai = -log1p(P->z_init);
  double dlna = -lnai / ns;
  t.a0 = (step == ns) ? 1.0 : exp(lnai + step * dlna);
  t.a1 = (step + 1 == ns) ? 1.0 : exp(lnai + (step + 1) * dlna);
  double ah = exp(lnai + (step + 0.5) * dlna);
  t.drift = dzso_drift_factor(P, t.a0, t.a1);
  t.kick1 = dzso_kick_factor(P, t.a0, ah);
  t.kick2 = dzso_kick_factor(P, ah, t.a1);
  double chi0 = dzso_chi(P, exp(lnai));
  t.rlc0 = rlc_of(P, t.a0, chi0);
  t.rlc1 = rlc_of(P, t.a1, chi0);
  t.rlat0 = (uint64_t)floor(t.rlc0 / P->box * 4294967296.0);
  t.rlat1 = (uint64_t)floor(t.rlc1 / P->box * 4294967296.0);
  return t;
}

static uint64_t dist2_obs(uint32_t x, uint32_t y, uint32_t z) {
  int64_t dx = (int32_t)(x - 2147483648u), dy = (int32_t)(y - 2147483648u),
          dz = (int32_t)(z - 2147483648u);
  return (uint64_t)(dx * dx) + (uint64_t)(dy * dy) + (uint64_t)(dz * dz);
}

void dzso_initial_flags(const dzso_params* P, int64_t n, const uint32_t* u, uint8_t* fl) {
  step_tab t = step_tables(P, 0);
  uint64_t r2 = t.rlat0 * t.rlat0;
  for (int64_t i = 0; i < n; ++i)
    if (dist2_obs(u[i], u[(size_t)n + i], u[2 * (size_t)n + i]) >= r2) fl[i] |= DZSO_FL_CROSSED;
}

int64_t dzso_kick_drift_cross(const dzso_params* P, int32_t step, int64_t n,
                              uint32_t* u, double* p, const double* g,
                              const uint32_t* k, const uint32_t* id, uint8_t* fl,
                              dzso_record* rec) {
  step_tab t = step_tables(P, step);
  double lat = 4294967296.0 / P->box;
  double scale = P->box / 4294967296.0;
  double dlat = t.drift * lat;
  uint64_t r20 = t.rlat0 * t.rlat0, r21 = t.rlat1 * t.rlat1;
  int64_t nrec = 0;
  for (int64_t i = 0; i < n; ++i) {
    uint32_t ub[3], ua[3];
    for (int ax = 0; ax < 3; ++ax) {
      size_t j = (size_t)ax * n + i;
      p[j] = p[j] + g[j] * t.kick1;
      ub[ax] = u[j];
      int64_t du = llrint(p[j] * dlat);
      ua[ax] = (uint32_t)((uint64_t)ub[ax] + (uint64_t)du);
      u[j] = ua[ax];
    }
    if (fl[i] & DZSO_FL_CROSSED) continue;
    uint64_t db = dist2_obs(ub[0], ub[1], ub[2]);
    uint64_t da = dist2_obs(ua[0], ua[1], ua[2]);
    if (db < r20 && da >= r21) {
      fl[i] |= DZSO_FL_CROSSED;
      if (rec) {
        double sb = sqrt((double)db) * scale - t.rlc0;
        double sa = sqrt((double)da) * scale - t.rlc1;
        double tt = sb / (sb - sa);
        if (!(tt >= 0.0)) tt = 0.0;
        if (tt > 1.0) tt = 1.0;
        dzso_record* r = &rec[nrec];
        r->id = id[i];
        r->k = k[i];
        r->a_cross = t.a0 + tt * (t.a1 - t.a0);
        for (int ax = 0; ax < 3; ++ax) {
          double x = (double)ub[ax] * scale + tt * (double)(int32_t)(ua[ax] - ub[ax]) * scale;
          if (x < 0.0) x += P->box;
          if (x >= P->box) x -= P->box;
          r->x[ax] = x;
          r->p[ax] = p[(size_t)ax * n + i];
        }
      }
      ++nrec;
    }
  }
  return nrec;
}

void dzso_accel(const dzso_params* P, int64_t n, const uint32_t* u,
                const uint32_t* k, double* g, int32_t parts,
                const int64_t* sample, int64_t nsample) {
  if (n == 0) return;
  uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
  int64_t* perm = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  int64_t* inv = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  dzso_sort(n, u, key, perm);
  uint32_t* su = (uint32_t*)malloc(sizeof(uint32_t) * 3 * (size_t)n);
  uint32_t* sk = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
  for (int64_t t = 0; t < n; ++t) {
    int64_t i = perm[t];
    inv[i] = t;
    for (int ax = 0; ax < 3; ++ax) su[(size_t)ax * n + t] = u[(size_t)ax * n + i];
    sk[t] = k[i];
  }
  int64_t* ssample = NULL;
  if (nsample > 0) {
    ssample = (int64_t*)malloc(sizeof(int64_t) * (size_t)nsample);
    for (int64_t s = 0; s < nsample; ++s) ssample[s] = inv[sample[s]];
  }
  double* gpm = (double*)calloc(3 * (size_t)n, sizeof(double));
  double* gtr = (double*)calloc(3 * (size_t)n, sizeof(double));
  if (parts & 1) {
    size_t m3 = (size_t)P->mesh * P->mesh * P->mesh;
    double* delta = (double*)malloc(sizeof(double) * m3);
    double* phi = (double*)malloc(sizeof(double) * m3);
    dzso_cic_delta(P, n, su, sk, delta);
    dzso_pm_potential(P, delta, phi);
    dzso_pm_accel(P, phi, n, su, gpm, ssample, nsample);
    free(delta);
    free(phi);
  }
  if (parts & 2) dzso_tree_accel(P, n, su, sk, gtr, ssample, nsample);
  for (int64_t t = 0; t < n; ++t) {
    int64_t i = perm[t];
    for (int ax = 0; ax < 3; ++ax)
      g[(size_t)ax * n + i] = gpm[(size_t)ax * n + t] + gtr[(size_t)ax * n + t];
  }
  free(gpm);
  free(gtr);
  free(ssample);
  free(su);
  free(sk);
  free(key);
  free(perm);
  free(inv);
}

int64_t dzso_step(const dzso_params* P, int32_t step, int64_t n, uint32_t* u,
                  double* p, double* g, uint32_t* k, uint32_t* id, uint8_t* fl,
                  dzso_record* rec, int64_t* nrec) {
  if (step < 0 || step >= P->nsteps) return -1;
  step_tab t = step_tables(P, step);
  int64_t nr = dzso_kick_drift_cross(P, step, n, u, p, g, k, id, fl, rec);
  if (nrec) *nrec = nr;
  /* a_old for the dynamical merge criterion: the previous accelerations of the
   * particles still inside the lightcone (g and fl share the pre-sort order) */
  double amin2 = dzso_amin2(n, g, fl);
  /* Morton sort, stable */
  uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
  int64_t* perm = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  dzso_sort(n, u, key, perm);
  uint32_t* tu = (uint32_t*)malloc(sizeof(uint32_t) * 3 * (size_t)(n > 0 ? n : 1));
  double* tp = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  uint32_t* tk = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
  uint32_t* tid = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
  uint8_t* tfl = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));
  for (int64_t s = 0; s < n; ++s) {
    int64_t i = perm[s];
    for (int ax = 0; ax < 3; ++ax) {
      tu[(size_t)ax * n + s] = u[(size_t)ax * n + i];
      tp[(size_t)ax * n + s] = p[(size_t)ax * n + i];
    }
    tk[s] = k[i];
    tid[s] = id[i];
    tfl[s] = fl[i];
  }
  memcpy(u, tu, sizeof(uint32_t) * 3 * (size_t)n);
  memcpy(p, tp, sizeof(double) * 3 * (size_t)n);
  memcpy(k, tk, sizeof(uint32_t) * (size_t)n);
  memcpy(id, tid, sizeof(uint32_t) * (size_t)n);
  memcpy(fl, tfl, (size_t)n);
  free(tu);
  free(tp);
  free(tk);
  free(tid);
  free(tfl);
  free(key);
  free(perm);
  if (P->dzs_on) n = dzso_merge(P, n, t.rlat1, amin2, u, p, k, id, fl);
  dzso_accel(P, n, u, k, g, 3, NULL, 0);
  for (size_t j = 0; j < 3 * (size_t)n; ++j) p[j] = p[j] + g[j] * t.kick2;
  return n;
}

void dzso_diagnostics(const dzso_params* P, int64_t n, const uint32_t* u,
                      const double* p, const uint32_t* k, double out[8]) {
  double scale = P->box / 4294967296.0;
  uint64_t K = 0, S[3] = {0, 0, 0};
  double pk[3] = {0.0, 0.0, 0.0};
  for (int64_t i = 0; i < n; ++i) {
    K += k[i];
    for (int ax = 0; ax < 3; ++ax) {
      S[ax] += (uint64_t)k[i] * u[(size_t)ax * n + i];
      pk[ax] += (double)k[i] * p[(size_t)ax * n + i];
    }
  }
  out[0] = (double)K;
  for (int ax = 0; ax < 3; ++ax) {
    out[1 + ax] = pk[ax];
    out[4 + ax] = (double)S[ax] * scale;
  }
  out[7] = (double)n;
}
