/*
 * tree.c -- oracle: Morton order, the oct-tree and the short-range tree force.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper's force tree is an oct-tree whose root is the box and whose nodes
 * are split into octants while they hold more than one particle; nodes carry
 * mass and centre of mass and the force uses their monopole only (Sec. 2.1).
 * A node is opened when l_n / d >= theta (Eq. 1).  The short-range force is
 * the Newtonian pair force times the TreePM split factor that matches the
 * exponential Fourier kernel of the PM part (Sec. 2.1):
 *   T(r) = erfc(r / 2 r_s) + r / (r_s sqrt(pi)) exp(-r^2 / 4 r_s^2),
 * set to zero beyond r_cut.  Readings where the paper is silent:
 *   - cells are the octree cells of the 21-bit-per-axis lattice prefix; a node
 *     is a leaf when it holds <= B particles or sits at depth 21;
 *   - the walk is done per group (node with <= G particles whose parent has
 *     more, or a leaf) against the group's cube: skip a node whose cube is
 *     farther than r_cut from the group cube, open it when the cubes touch or
 *     l_n >= theta d(COM_n, group cube), else use its monopole; a monopole or
 *     a particle of an opened leaf that lies farther than r_cut from the group
 *     cube is left off the list (it is farther than r_cut from every particle
 *     of the group, so its short-range force on them is zero);
 *   - softening: cubic-spline kernel of Plummer-equivalent eps
 *     (spline radius 2.8 eps), eps = eps0 k^(1/3) (Sec. 2.2 rescaling),
 *     pair softening max(eps_i, eps_j), node softening = max over members;
 *   - node COM = floor((2 S + K) / (2 K)) per axis on the integer lattice,
 *     S = sum k u, K = sum k (exact).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

/* ---------------- Morton keys and the stable sort ---------------- */

uint64_t dzso_morton_key(uint32_t ux, uint32_t uy, uint32_t uz) {
  uint32_t x = ux >> 11, y = uy >> 11, z = uz >> 11;
  uint64_t key = 0;
  for (int b = 0; b < 21; ++b) {
    key |= (uint64_t)((x >> b) & 1u) << (3 * b + 2);
    key |= (uint64_t)((y >> b) & 1u) << (3 * b + 1);
    key |= (uint64_t)((z >> b) & 1u) << (3 * b);
  }
  return key;
}

static const uint64_t* g_sort_keys; /* comparator context (single-threaded sort) */

static int cmp_key_then_index(const void* a, const void* b) {
  int64_t ia = *(const int64_t*)a, ib = *(const int64_t*)b;
  uint64_t ka = g_sort_keys[ia], kb = g_sort_keys[ib];
  if (ka != kb) return ka < kb ? -1 : 1;
  return ia < ib ? -1 : (ia > ib ? 1 : 0);
}

/* keys in input order and the stable ascending permutation:
 * sorted position t holds input particle perm[t] */
void dzso_sort(int64_t n, const uint32_t* u, uint64_t* key, int64_t* perm) {
  for (int64_t i = 0; i < n; ++i) {
    key[i] = dzso_morton_key(u[i], u[(size_t)n + i], u[2 * (size_t)n + i]);
    perm[i] = i;
  }
  g_sort_keys = key;
  qsort(perm, (size_t)n, sizeof(int64_t), cmp_key_then_index);
}

/* ---------------- explicit oct-tree over sorted particles ---------------- */

typedef struct {
  int level;
  int64_t s, e;          /* particle range [s, e) */
  uint64_t center[3];    /* cube centre on the lattice */
  uint64_t side;         /* 2^(32 - level) */
  uint64_t K;            /* sum k */
  uint32_t com[3];       /* rounded integer centre of mass */
  uint32_t kmax;         /* largest member multiplicity */
  int64_t child;         /* first child node, -1 for a leaf */
  int nchild;
} onode;

typedef struct {
  onode* nodes;
  int64_t count, cap;
} otree;

static int64_t tree_alloc(otree* t, int64_t k) {
  if (t->count + k > t->cap) {
    t->cap = (t->count + k) * 2 + 64;
    t->nodes = (onode*)realloc(t->nodes, sizeof(onode) * (size_t)t->cap);
  }
  int64_t r = t->count;
  t->count += k;
  return r;
}

static int digit_at(uint64_t key, int level) { /* level >= 1 */
  return (int)((key >> (3 * (21 - level))) & 7u);
}

static void fill_node(onode* nd, int level, int64_t s, int64_t e, int64_t n,
                      const uint32_t* u, const uint32_t* k) {
  nd->level = level;
  nd->s = s;
  nd->e = e;
  nd->side = 1ull << (32 - level);
  for (int ax = 0; ax < 3; ++ax) {
    uint64_t origin = 0;
    if (level > 0) origin = ((uint64_t)u[(size_t)ax * n + s] >> (32 - level)) << (32 - level);
    nd->center[ax] = origin + nd->side / 2;
  }
  uint64_t K = 0, S[3] = {0, 0, 0};
  uint32_t kmax = 0;
  for (int64_t i = s; i < e; ++i) {
    K += k[i];
    for (int ax = 0; ax < 3; ++ax) S[ax] += (uint64_t)k[i] * u[(size_t)ax * n + i];
    if (k[i] > kmax) kmax = k[i];
  }
  nd->K = K;
  nd->kmax = kmax;
  for (int ax = 0; ax < 3; ++ax) nd->com[ax] = (uint32_t)((2 * S[ax] + K) / (2 * K));
  nd->child = -1;
  nd->nchild = 0;
}

static void build_rec(otree* t, int64_t idx, const uint64_t* key, int64_t n,
                      const uint32_t* u, const uint32_t* k, int B) {
  onode nd = t->nodes[idx];
  if (nd.e - nd.s <= B || nd.level == 21) return;
  /* children in octant order: consecutive runs of the next digit */
  int64_t cs[8], ce[8];
  int nc = 0;
  int64_t i = nd.s;
  while (i < nd.e) {
    int d = digit_at(key[i], nd.level + 1);
    int64_t j = i;
    while (j < nd.e && digit_at(key[j], nd.level + 1) == d) ++j;
    cs[nc] = i;
    ce[nc] = j;
    ++nc;
    i = j;
  }
  int64_t first = tree_alloc(t, nc);
  t->nodes[idx].child = first;
  t->nodes[idx].nchild = nc;
  for (int c = 0; c < nc; ++c) fill_node(&t->nodes[first + c], nd.level + 1, cs[c], ce[c], n, u, k);
  for (int c = 0; c < nc; ++c) build_rec(t, first + c, key, n, u, k, B);
}

static otree build_tree(const dzso_params* P, int64_t n, const uint32_t* u, const uint32_t* k) {
  otree t = {NULL, 0, 0};
  uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) key[i] = dzso_morton_key(u[i], u[(size_t)n + i], u[2 * (size_t)n + i]);
  tree_alloc(&t, 1);
  fill_node(&t.nodes[0], 0, 0, n, n, u, k);
  build_rec(&t, 0, key, n, u, k, P->leaf_bucket);
  free(key);
  return t;
}

/* groups: descend from the root while the node has > G particles and is not a
 * leaf; the node reached is a group */
static void groups_rec(const otree* t, int64_t idx, int G, int64_t* out, int64_t* ng) {
  const onode* nd = &t->nodes[idx];
  if (nd->e - nd->s <= G || nd->child < 0) {
    if (out) out[*ng] = idx;
    ++*ng;
    return;
  }
  for (int c = 0; c < nd->nchild; ++c) groups_rec(t, nd->child + c, G, out, ng);
}

/* ---------------- pair force ---------------- */

/* cubic-spline softened 1/r^3 (kernel of Monaghan & Lattanzio 1985 integrated
 * for the enclosed mass m(u), u = r/h: fac = m(u) / r^3) times the TreePM
 * short-range factor T(r) */
double dzso_pair_factor(const dzso_params* P, double r, double h) {
  double rs = P->rs_cells * P->box / P->mesh;
  double fac;
  if (r >= h) {
    fac = 1.0 / (r * r * r);
  } else {
    double q = r / h, h3 = h * h * h;
    if (q < 0.5)
      fac = (32.0 / 3.0 - 192.0 / 5.0 * q * q + 32.0 * q * q * q) / h3;
    else
      fac = (64.0 / 3.0 - 48.0 * q + 192.0 / 5.0 * q * q - 32.0 / 3.0 * q * q * q -
             1.0 / 15.0 / (q * q * q)) / h3;
  }
  double t = erfc(r / (2.0 * rs)) + r / (rs * sqrt(M_PI)) * exp(-r * r / (4.0 * rs * rs));
  return fac * t;
}

typedef struct {
  uint32_t x[3];
  uint32_t k, kmax;
} lentry;

typedef struct {
  lentry* e;
  int64_t n, cap;
} llist;

static void list_push(llist* l, const uint32_t x[3], uint32_t k, uint32_t kmax) {
  if (l->n == l->cap) {
    l->cap = l->cap * 2 + 256;
    l->e = (lentry*)realloc(l->e, sizeof(lentry) * (size_t)l->cap);
  }
  lentry* q = &l->e[l->n++];
  q->x[0] = x[0];
  q->x[1] = x[1];
  q->x[2] = x[2];
  q->k = k;
  q->kmax = kmax;
}

static int64_t iabs64(int64_t v) { return v < 0 ? -v : v; }

/* squared lattice distance from point x to the group cube (centre cg, side lg) */
static uint64_t point_cube_d2(const uint32_t x[3], const uint64_t cg[3], uint64_t lg) {
  uint64_t d2 = 0;
  for (int ax = 0; ax < 3; ++ax) {
    int64_t dm = iabs64((int64_t)(int32_t)(uint32_t)((uint64_t)x[ax] - cg[ax])) - (int64_t)(lg / 2);
    if (dm > 0) d2 += (uint64_t)dm * (uint64_t)dm;
  }
  return d2;
}

/* depth-first walk of node idx for the group cube (cg, lg) */
static void walk_rec(const dzso_params* P, const otree* t, int64_t idx, const uint64_t cg[3],
                     uint64_t lg, double rcut_lat2, int64_t n, const uint32_t* u,
                     const uint32_t* k, llist* out) {
  const onode* nd = &t->nodes[idx];
  int touch = 1;
  uint64_t dist2 = 0, dcom2 = 0;
  for (int ax = 0; ax < 3; ++ax) {
    int64_t dc = iabs64((int64_t)(int32_t)(uint32_t)(nd->center[ax] - cg[ax]));
    int64_t gap = dc - (int64_t)((lg + nd->side) / 2);
    if (gap > 0) {
      touch = 0;
      dist2 += (uint64_t)gap * (uint64_t)gap;
    }
    int64_t dm = iabs64((int64_t)(int32_t)(uint32_t)((uint64_t)nd->com[ax] - cg[ax])) - (int64_t)(lg / 2);
    if (dm > 0) dcom2 += (uint64_t)dm * (uint64_t)dm;
  }
  if (!touch && (double)dist2 > rcut_lat2) return; /* every pair beyond r_cut */
  int open = touch || ((double)nd->side >= P->theta * sqrt((double)dcom2));
  if (!open) {
    /* a monopole farther than r_cut from the group cube acts on none of the
     * group's particles: not listed */
    if ((double)dcom2 <= rcut_lat2) list_push(out, nd->com, (uint32_t)nd->K, nd->kmax);
    return;
  }
  if (nd->child < 0) {
    for (int64_t i = nd->s; i < nd->e; ++i) {
      uint32_t x[3] = {u[i], u[(size_t)n + i], u[2 * (size_t)n + i]};
      /* likewise a particle of an opened leaf farther than r_cut from the
       * group cube (same distance rule as the node skip) */
      if ((double)point_cube_d2(x, cg, lg) > rcut_lat2) continue;
      list_push(out, x, k[i], k[i]);
    }
    return;
  }
  for (int c = 0; c < nd->nchild; ++c) walk_rec(P, t, nd->child + c, cg, lg, rcut_lat2, n, u, k, out);
}

typedef struct {
  double scale, gm0, eps0, rcut2;
} force_consts;

static force_consts make_consts(const dzso_params* P) {
  force_consts c;
  double n0 = (double)P->n1d * P->n1d * P->n1d;
  double rs = P->rs_cells * P->box / P->mesh;
  double rcut = P->rcut_rs * rs;
  c.scale = P->box / 4294967296.0;
  c.gm0 = 1.5 * P->omega_m * P->box * P->box * P->box / (4.0 * M_PI * n0);
  c.eps0 = P->soft_frac * P->box / P->n1d;
  c.rcut2 = rcut * rcut;
  return c;
}

static void eval_particle(const dzso_params* P, const force_consts* c, const llist* l,
                          int64_t n, const uint32_t* u, const uint32_t* k, int64_t i,
                          double* g) {
  double acc[3] = {0.0, 0.0, 0.0};
  double epsi = c->eps0 * cbrt((double)k[i]);
  uint32_t xi[3] = {u[i], u[(size_t)n + i], u[2 * (size_t)n + i]};
  for (int64_t e = 0; e < l->n; ++e) {
    const lentry* q = &l->e[e];
    double d[3];
    for (int ax = 0; ax < 3; ++ax) d[ax] = (double)(int32_t)(q->x[ax] - xi[ax]) * c->scale;
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2 == 0.0 || r2 >= c->rcut2) continue;
    double r = sqrt(r2);
    double epsj = c->eps0 * cbrt((double)q->kmax);
    double h = 2.8 * (epsi > epsj ? epsi : epsj);
    double f = c->gm0 * (double)q->k * dzso_pair_factor(P, r, h);
    for (int ax = 0; ax < 3; ++ax) acc[ax] += f * d[ax];
  }
  for (int ax = 0; ax < 3; ++ax) g[(size_t)ax * n + i] = acc[ax];
}

static double rcut_lattice2(const dzso_params* P) {
  double rs = P->rs_cells * P->box / P->mesh;
  double rcut_lat = P->rcut_rs * rs / P->box * 4294967296.0;
  return rcut_lat * rcut_lat;
}

void dzso_tree_accel(const dzso_params* P, int64_t n, const uint32_t* u,
                     const uint32_t* k, double* g, const int64_t* sample,
                     int64_t nsample) {
  if (n == 0) return;
  otree t = build_tree(P, n, u, k);
  int64_t ng = 0;
  groups_rec(&t, 0, P->walk_group, NULL, &ng);
  int64_t* groups = (int64_t*)malloc(sizeof(int64_t) * (size_t)ng);
  ng = 0;
  groups_rec(&t, 0, P->walk_group, groups, &ng);
  unsigned char* want = NULL;
  unsigned char* gwant = (unsigned char*)calloc((size_t)ng, 1);
  if (nsample > 0) {
    want = (unsigned char*)calloc((size_t)n, 1);
    for (int64_t s = 0; s < nsample; ++s) want[sample[s]] = 1;
    for (int64_t gi = 0; gi < ng; ++gi) {
      const onode* nd = &t.nodes[groups[gi]];
      for (int64_t i = nd->s; i < nd->e; ++i)
        if (want[i]) gwant[gi] = 1;
    }
  } else {
    memset(gwant, 1, (size_t)ng);
  }
  force_consts c = make_consts(P);
  double rl2 = rcut_lattice2(P);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t gi = 0; gi < ng; ++gi) {
    if (!gwant[gi]) continue;
    const onode* gn = &t.nodes[groups[gi]];
    llist l = {NULL, 0, 0};
    walk_rec(P, &t, 0, gn->center, gn->side, rl2, n, u, k, &l);
    for (int64_t i = gn->s; i < gn->e; ++i)
      if (!want || want[i]) eval_particle(P, &c, &l, n, u, k, i, g);
    free(l.e);
  }
  free(want);
  free(gwant);
  free(groups);
  free(t.nodes);
}

/* number of groups; optional outputs of their particle ranges */
int64_t dzso_count_groups(const dzso_params* P, int64_t n, const uint32_t* u,
                          int64_t* group_start, int64_t* group_count) {
  if (n == 0) return 0;
  uint32_t* ones = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) ones[i] = 1;
  otree t = build_tree(P, n, u, ones);
  int64_t ng = 0;
  groups_rec(&t, 0, P->walk_group, NULL, &ng);
  int64_t* groups = (int64_t*)malloc(sizeof(int64_t) * (size_t)ng);
  ng = 0;
  groups_rec(&t, 0, P->walk_group, groups, &ng);
  for (int64_t gi = 0; gi < ng; ++gi) {
    if (group_start) group_start[gi] = t.nodes[groups[gi]].s;
    if (group_count) group_count[gi] = t.nodes[groups[gi]].e - t.nodes[groups[gi]].s;
  }
  free(groups);
  free(t.nodes);
  free(ones);
  return ng;
}

/* length of the interaction list of one group (group_index >= 0), or the total
 * number of particle-entry pairs evaluated over all groups (group_index < 0) */
int64_t dzso_interaction_count(const dzso_params* P, int64_t n, const uint32_t* u,
                               const uint32_t* k, int64_t group_index) {
  if (n == 0) return 0;
  otree t = build_tree(P, n, u, k);
  int64_t ng = 0;
  groups_rec(&t, 0, P->walk_group, NULL, &ng);
  int64_t* groups = (int64_t*)malloc(sizeof(int64_t) * (size_t)ng);
  ng = 0;
  groups_rec(&t, 0, P->walk_group, groups, &ng);
  double rl2 = rcut_lattice2(P);
  int64_t total = 0;
  for (int64_t gi = 0; gi < ng; ++gi) {
    if (group_index >= 0 && gi != group_index) continue;
    const onode* gn = &t.nodes[groups[gi]];
    llist l = {NULL, 0, 0};
    walk_rec(P, &t, 0, gn->center, gn->side, rl2, n, u, k, &l);
    total += (group_index >= 0) ? l.n : l.n * (gn->e - gn->s);
    free(l.e);
  }
  free(groups);
  free(t.nodes);
  return total;
}
