/*
 * fof.c -- oracle: friends-of-friends haloes.  TEST INFRASTRUCTURE ONLY (see
 * oracle.h).
 *
 * Paper Sec. 3.1.1: the lightcone halo mass function is built from the FoF
 * halo catalogues of frequent outputs (the FoF finder of the simulation code),
 * keeping the haloes entirely inside the lightcone at the time of each output.
 * Reading (the paper gives no linking length): two particles are
 * friends when their minimum-image lattice distance satisfies
 *     d^2 <= T,   T = floor((link * 2^32 / n1d)^2)   (FP64, then integer),
 * i.e. d <= link * lambda with lambda = L / n1d the initial mean spacing; a
 * halo is a connected component of the friends graph with at least nmin
 * particles.  Each halo reports: its first particle (the smallest index, which
 * also labels every member), its particle count, its mass sum k, its centre of
 * mass x = (u_first + S / K) L / 2^32 wrapped into [0, L) with S = sum k
 * (u - u_first) over members (minimum-image offsets, exact int64) and K = sum
 * k, and the largest squared lattice distance of a member from the observer
 * (for the "entirely inside the lightcone" test).
 *
 * Neighbours: all pairs for n <= 4096; otherwise a uniform grid of 2^D cells
 * per side with cell side 2^(32-D) >= the linking length, scanning the 27
 * neighbour cells (the union-find result does not depend on the scan).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

static int64_t uf_find(int64_t* par, int64_t x) {
  while (par[x] != x) {
    par[x] = par[par[x]];
    x = par[x];
  }
  return x;
}

static void uf_union(int64_t* par, int64_t a, int64_t b) {
  a = uf_find(par, a);
  b = uf_find(par, b);
  if (a == b) return;
  if (a < b)
    par[b] = a;
  else
    par[a] = b;
}

static uint64_t pair_d2(const uint32_t* u, int64_t n, int64_t i, int64_t j) {
  uint64_t d2 = 0;
  for (int ax = 0; ax < 3; ++ax) {
    int64_t d = (int32_t)(u[(size_t)ax * n + j] - u[(size_t)ax * n + i]);
    d2 += (uint64_t)(d * d);
  }
  return d2;
}

uint64_t dzso_fof_threshold(const dzso_params* P, double link) {
  double lb = link * 4294967296.0 / (double)P->n1d;
  return (uint64_t)floor(lb * lb);
}

typedef struct {
  int64_t cell;
  int64_t idx;
} cell_item;

static int cmp_item(const void* a, const void* b) {
  const cell_item* x = (const cell_item*)a;
  const cell_item* y = (const cell_item*)b;
  if (x->cell != y->cell) return x->cell < y->cell ? -1 : 1;
  return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

int64_t dzso_fof(const dzso_params* P, int64_t n, const uint32_t* u, const uint32_t* k, double link, int32_t nmin,
                 int64_t* label, dzso_halo* halos) {
  const uint64_t T = dzso_fof_threshold(P, link);
  int64_t* par = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) par[i] = i;
  if (n <= 4096) {
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = i + 1; j < n; ++j)
        if (pair_d2(u, n, i, j) <= T) uf_union(par, i, j);
  } else {
    /* cells of side 2^(32 - D) >= sqrt(T) */
    int D = 1;
    while (D < 10 && ldexp(1.0, 32 - (D + 1)) * ldexp(1.0, 32 - (D + 1)) >= (double)T + 1.0) ++D;
    const int64_t nc = (int64_t)1 << D;
    cell_item* it = (cell_item*)malloc(sizeof(cell_item) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
      int64_t cx = u[i] >> (32 - D), cy = u[(size_t)n + i] >> (32 - D), cz = u[2 * (size_t)n + i] >> (32 - D);
      it[i].cell = (cx * nc + cy) * nc + cz;
      it[i].idx = i;
    }
    qsort(it, (size_t)n, sizeof(cell_item), cmp_item);
    int64_t* start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nc * nc * nc + 1));
    for (int64_t c = 0, p = 0; c <= nc * nc * nc; ++c) {
      while (p < n && it[p].cell < c) ++p;
      start[c] = p;
    }
    for (int64_t i = 0; i < n; ++i) {
      int64_t cx = u[i] >> (32 - D), cy = u[(size_t)n + i] >> (32 - D), cz = u[2 * (size_t)n + i] >> (32 - D);
      for (int ox = -1; ox <= 1; ++ox)
        for (int oy = -1; oy <= 1; ++oy)
          for (int oz = -1; oz <= 1; ++oz) {
            int64_t c = ((((cx + ox) % nc + nc) % nc) * nc + (((cy + oy) % nc + nc) % nc)) * nc +
                        (((cz + oz) % nc + nc) % nc);
            for (int64_t p = start[c]; p < start[c + 1]; ++p) {
              int64_t j = it[p].idx;
              if (j > i && pair_d2(u, n, i, j) <= T) uf_union(par, i, j);
            }
          }
    }
    free(start);
    free(it);
  }
  /* components: roots are the smallest member index */
  int64_t* cnt = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) {
    par[i] = uf_find(par, i);
    cnt[par[i]] += 1;
  }
  int64_t nh = 0;
  int64_t* hid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) {
    hid[i] = -1;
    if (par[i] == i && cnt[i] >= nmin) {
      hid[i] = nh;
      dzso_halo* h = &halos[nh++];
      memset(h, 0, sizeof(*h));
      h->first = i;
      h->count = cnt[i];
    }
  }
  int64_t* S = (int64_t*)calloc((size_t)(nh > 0 ? nh : 1) * 3, sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) {
    int64_t r = par[i];
    int64_t h = hid[r];
    if (label) label[i] = h >= 0 ? r : -1;
    if (h < 0) continue;
    dzso_halo* H = &halos[h];
    H->mass += k[i];
    for (int ax = 0; ax < 3; ++ax)
      S[3 * h + ax] += (int64_t)k[i] * (int64_t)(int32_t)(u[(size_t)ax * n + i] - u[(size_t)ax * n + r]);
    uint64_t d2 = 0;
    for (int ax = 0; ax < 3; ++ax) {
      int64_t o = (int32_t)(u[(size_t)ax * n + i] - 2147483648u);
      d2 += (uint64_t)(o * o);
    }
    if (d2 > H->rmax2) H->rmax2 = d2;
  }
  const double scale = P->box / 4294967296.0;
  for (int64_t h = 0; h < nh; ++h) {
    dzso_halo* H = &halos[h];
    for (int ax = 0; ax < 3; ++ax) {
      double x = ((double)u[(size_t)ax * n + H->first] + (double)S[3 * h + ax] / (double)H->mass) * scale;
      if (x < 0.0) x += P->box;
      if (x >= P->box) x -= P->box;
      H->x[ax] = x;
    }
  }
  free(S);
  free(hid);
  free(cnt);
  free(par);
  return nh;
}
