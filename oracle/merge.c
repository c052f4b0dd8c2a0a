/*
 * merge.c -- oracle: the DZS de-refinement walk.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Paper, Sec. 2.2 and Fig. 2: the oct-tree is walked once from the root; a
 * node that meets the merge criteria is replaced by one particle carrying its
 * centre-of-mass properties (mass, position, velocity), otherwise the walk
 * continues into its children.  Sec. 2.2.1: the criterion is the geometric
 * opening rule with d replaced by the node distance of Eq. 3,
 *   D_n = max(d_{n-obs} - R_lc - b, 0),   merge iff l_n / D_n < theta_dzs,
 * with node sizes limited to l_n <= l_max (Sec. 2.2).  Readings where the
 * paper is silent:
 *   - cells are octree cells of side L / 2^j down to depth 21; a cell with a
 *     single particle is left alone; l_max = 2^(merge_level-1) lambda;
 *   - integer test: merge iff d_COM^2 > T^2, T = R_lat + b_lat + ceil(l_lat /
 *     theta_dzs) (lattice units; T >= 2^32 never merges);
 *   - dynamical criterion (Sec. 2.2.1: Eq. 2 with d -> D_n of Eq. 3 and
 *     |a_old| -> the smallest |a| of the particles inside the lightcone, i.e.
 *     not yet crossed): merge iff D > 0 and G M_n l^2 / D^4 < alpha a_min,
 *     D = (sqrt(d_COM^2) - R_lat - b_lat) L / 2^32, in FP64 in this order;
 *   - new particle: k = sum k, u = floor((2 S + K) / (2 K)), p = (sum k p) / K
 *     with the FP64 sum taken left to right in Morton order, id = min id,
 *     flags = merged | crossed.  The survivors keep their Morton order.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

/* coarsest level whose cell side L / 2^j is <= l_max = 2^(ell-1) L / n1d,
 * i.e. the smallest j >= 1 with 2^j 2^(ell-1) >= n1d */
int32_t dzso_merge_jmin(const dzso_params* P) {
  int32_t j = 1;
  while (((int64_t)1 << j) * ((int64_t)1 << (P->merge_level - 1)) < P->n1d) ++j;
  return j;
}

uint64_t dzso_merge_threshold(const dzso_params* P, uint64_t rlat, int32_t level) {
  double lat = 4294967296.0;
  uint64_t blat = (uint64_t)floor(P->buffer_cells * lat / P->mesh);
  double lovt = ceil(ldexp(1.0, 32 - level) / P->theta_dzs);
  if (!(lovt < lat)) return UINT64_MAX;
  uint64_t t = rlat + blat + (uint64_t)lovt;
  return t;
}

typedef struct {
  const dzso_params* P;
  int64_t n;
  uint64_t rlat;
  double amin2;
  int32_t jmin;
  const uint64_t* key;
  const uint32_t* u;
  const double* p;
  const uint32_t* k;
  const uint32_t* id;
  const uint8_t* fl;
  /* output */
  uint32_t* ou;
  double* op;
  uint32_t* ok;
  uint32_t* oid;
  uint8_t* ofl;
  int64_t nout;
} mctx;

static void keep_one(mctx* c, int64_t i) {
  int64_t o = c->nout++;
  for (int ax = 0; ax < 3; ++ax) {
    c->ou[(size_t)ax * c->n + o] = c->u[(size_t)ax * c->n + i];
    c->op[(size_t)ax * c->n + o] = c->p[(size_t)ax * c->n + i];
  }
  c->ok[o] = c->k[i];
  c->oid[o] = c->id[i];
  c->ofl[o] = c->fl[i];
}

static int qualifies_dynamical(mctx* c, int level, uint64_t K, const uint32_t com[3]) {
  const dzso_params* P = c->P;
  double lat = 4294967296.0;
  uint64_t blat = (uint64_t)floor(P->buffer_cells * lat / P->mesh);
  uint64_t d2 = 0;
  for (int ax = 0; ax < 3; ++ax) {
    int64_t off = (int64_t)(int32_t)(com[ax] - 2147483648u);
    d2 += (uint64_t)(off * off);
  }
  double scale = P->box / lat;
  double D = (sqrt((double)d2) - (double)(c->rlat + blat)) * scale;
  if (!(D > 0.0)) return 0;
  double n0 = (double)P->n1d * P->n1d * P->n1d;
  double gm0 = 1.5 * P->omega_m * P->box * P->box * P->box / (4.0 * M_PI * n0);
  double l = ldexp(P->box, -level);
  double D2 = D * D;
  double lhs = gm0 * (double)K * (l * l) / (D2 * D2);
  double rhs = P->alpha_dyn * sqrt(c->amin2);
  return lhs < rhs;
}

static int qualifies(mctx* c, int level, int64_t s, int64_t e, uint64_t K, const uint32_t com[3]) {
  (void)s;
  (void)e;
  if (c->P->criterion == 1) return qualifies_dynamical(c, level, K, com);
  uint64_t t = dzso_merge_threshold(c->P, c->rlat, level);
  if (t >= 4294967296ull) return 0;
  uint64_t d2 = 0;
  for (int ax = 0; ax < 3; ++ax) {
    int64_t off = (int64_t)(int32_t)(com[ax] - 2147483648u);
    d2 += (uint64_t)(off * off);
  }
  return d2 > t * t;
}

static void merge_cell(mctx* c, int level, int64_t s, int64_t e) {
  int64_t cnt = e - s;
  if (cnt == 1) {
    keep_one(c, s);
    return;
  }
  if (level >= c->jmin) {
    uint64_t K = 0, S[3] = {0, 0, 0};
    for (int64_t i = s; i < e; ++i) {
      K += c->k[i];
      for (int ax = 0; ax < 3; ++ax) S[ax] += (uint64_t)c->k[i] * c->u[(size_t)ax * c->n + i];
    }
    uint32_t com[3];
    for (int ax = 0; ax < 3; ++ax) com[ax] = (uint32_t)((2 * S[ax] + K) / (2 * K));
    if (qualifies(c, level, s, e, K, com)) {
      int64_t o = c->nout++;
      uint32_t idmin = c->id[s];
      for (int ax = 0; ax < 3; ++ax) {
        double sum = 0.0;
        for (int64_t i = s; i < e; ++i) sum += (double)c->k[i] * c->p[(size_t)ax * c->n + i];
        c->op[(size_t)ax * c->n + o] = sum / (double)K;
        c->ou[(size_t)ax * c->n + o] = com[ax];
      }
      for (int64_t i = s; i < e; ++i)
        if (c->id[i] < idmin) idmin = c->id[i];
      c->ok[o] = (uint32_t)K;
      c->oid[o] = idmin;
      c->ofl[o] = (uint8_t)(DZSO_FL_MERGED | DZSO_FL_CROSSED);
      return;
    }
  }
  if (level == 21) {
    for (int64_t i = s; i < e; ++i) keep_one(c, i);
    return;
  }
  /* children: runs of equal digit at level + 1 */
  int64_t i = s;
  while (i < e) {
    int shift = 3 * (21 - (level + 1));
    uint64_t d = (c->key[i] >> shift) & 7u;
    int64_t j = i;
    while (j < e && ((c->key[j] >> shift) & 7u) == d) ++j;
    merge_cell(c, level + 1, i, j);
    i = j;
  }
}

double dzso_amin2(int64_t n, const double* g, const uint8_t* fl) {
  double m = INFINITY;
  for (int64_t i = 0; i < n; ++i) {
    if (fl[i] & DZSO_FL_CROSSED) continue;
    double gx = g[i], gy = g[(size_t)n + i], gz = g[2 * (size_t)n + i];
    double a2 = gx * gx + gy * gy + gz * gz;
    if (a2 < m) m = a2;
  }
  return m;
}

int64_t dzso_merge(const dzso_params* P, int64_t n, uint64_t rlat, double amin2, uint32_t* u,
                   double* p, uint32_t* k, uint32_t* id, uint8_t* fl) {
  if (n == 0) return 0;
  uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) key[i] = dzso_morton_key(u[i], u[(size_t)n + i], u[2 * (size_t)n + i]);
  mctx c;
  memset(&c, 0, sizeof(c));
  c.P = P;
  c.n = n;
  c.rlat = rlat;
  c.amin2 = amin2;
  c.jmin = dzso_merge_jmin(P);
  c.key = key;
  c.u = u;
  c.p = p;
  c.k = k;
  c.id = id;
  c.fl = fl;
  c.ou = (uint32_t*)malloc(sizeof(uint32_t) * 3 * (size_t)n);
  c.op = (double*)malloc(sizeof(double) * 3 * (size_t)n);
  c.ok = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
  c.oid = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
  c.ofl = (uint8_t*)malloc((size_t)n);
  merge_cell(&c, 0, 0, n);
  int64_t m = c.nout;
  /* write back compactly: SoA with stride m */
  for (int ax = 0; ax < 3; ++ax)
    for (int64_t i = 0; i < m; ++i) {
      u[(size_t)ax * m + i] = c.ou[(size_t)ax * n + i];
      p[(size_t)ax * m + i] = c.op[(size_t)ax * n + i];
    }
  memcpy(k, c.ok, sizeof(uint32_t) * (size_t)m);
  memcpy(id, c.oid, sizeof(uint32_t) * (size_t)m);
  memcpy(fl, c.ofl, (size_t)m);
  free(c.ou);
  free(c.op);
  free(c.ok);
  free(c.oid);
  free(c.ofl);
  free(key);
  return m;
}
