/*
 * oracle.h -- plain, slow FP64 CPU oracle of one DZS TreePM KDK step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: only tests/, the smoke check and the benchmark's CPU-baseline
 * leg use it.  It shares no code, header, table or constant generator with the
 * CUDA library (include/dzs.h, paper_2005_05328_gb300/csrc/).
 *
 * What it computes (paper: Garaldi, Nori & Baldi, "Dynamic Zoom Simulations",
 * arXiv 2005.05328):
 *   - TreePM gravity: PM long-range force with a Gaussian split combined in
 *     Fourier space (Sec. 2.1) and a monopole-only short-range oct-tree force
 *     (Sec. 2.1) opened with the geometric criterion (Eq. 1);
 *   - softening rescaled by (M/M_init)^(1/3) (Sec. 2.2);
 *   - the DZS top-down merge walk (Sec. 2.2, Fig. 2) with the node distance of
 *     Eq. 3 and the geometric criterion l_n / D_n < theta (Sec. 2.2.1);
 *   - the lightcone shell crossing at R_lc(a) (Sec. 1 footnote, Sec. 3.1.3);
 *   - global KDK steps (Sec. 2.1: DZS runs only on global steps).
 * Where the paper is silent the oracle takes its own stated readings (lattice
 * positions, ICs, cubic-spline softening, group walk, ...), each written out in
 * the file that implements it.
 *
 * Parity status: every function below is pinned by tests/test_oracle_*.py
 * against closed forms, brute force or invariants, except
 * dzso_step's multi-step trajectories (chaotic; checked statistically).
 *
 * Conventions
 *   positions: uint32 lattice u = floor(x / L * 2^32) per axis, SoA [3][n];
 *              periodic wrap is uint32 overflow; observer at u = 2^31.
 *   masses:    uint32 multiplicity k, physical mass k * m0.
 *   units:     H0 = 1, lengths in Mpc/h, canonical momentum p = a^2 dx/dt.
 *   flags:     bit 0 crossed the lightcone, bit 1 product of a merge.
 */
#ifndef DZSO_ORACLE_H
#define DZSO_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#define DZSO_FL_CROSSED 1u
#define DZSO_FL_MERGED 2u

#define DZSO_RLC_SWEEP 0
#define DZSO_RLC_PHYSICAL 1

typedef struct {
  int32_t n1d;          /* particles per side at the start, N0 = n1d^3 */
  int32_t mesh;         /* PM mesh points per side M */
  double box;           /* L [Mpc/h] */
  double omega_m, omega_l, hubble, sigma8, ns;
  double z_init;
  int32_t nsteps;       /* global KDK steps, uniform in ln a to a = 1 */
  int32_t leaf_bucket;  /* B: tree leaf holds <= B particles */
  int32_t walk_group;   /* G: walk group = node with <= G particles, parent > G */
  int32_t dzs_on;
  int32_t merge_level;  /* l_max = 2^(merge_level-1) * lambda */
  int32_t rlc_mode;     /* DZSO_RLC_SWEEP | DZSO_RLC_PHYSICAL */
  double rs_cells;      /* r_s in mesh cells */
  double rcut_rs;       /* r_cut / r_s */
  double theta;         /* force-walk opening angle (Eq. 1) */
  double soft_frac;     /* eps0 / lambda */
  double theta_dzs;     /* DZS geometric merge angle (Sec. 2.2.1) */
  double buffer_cells;  /* buffer b in mesh cells (Eq. 3) */
  uint64_t seed;
  int32_t criterion;    /* 0: geometric l/D < theta_dzs; 1: dynamical (Eq. 2 with D of Eq. 3) */
  int32_t pad_;
  double alpha_dyn;     /* dynamical merge parameter alpha */
} dzso_params;

typedef struct {
  uint32_t id, k;
  double a_cross;
  double x[3];
  double p[3];
} dzso_record;

/* ---- cosmology (cosmo.c) ---- */
double dzso_hubble_e(const dzso_params* P, double a);
double dzso_drift_factor(const dzso_params* P, double a0, double a1);
double dzso_kick_factor(const dzso_params* P, double a0, double a1);
double dzso_chi(const dzso_params* P, double a);
double dzso_growth(const dzso_params* P, double a);       /* D+(a), D+(1) = 1 */
double dzso_growth_rate(const dzso_params* P, double a);  /* f = dlnD+/dlna */
double dzso_power(const dzso_params* P, double k);         /* normalised to sigma8 */
double dzso_power_amplitude(const dzso_params* P);         /* A in P = A k^ns T^2 */
double dzso_power_shape(const dzso_params* P, double k);   /* k^ns T^2 */
double dzso_sigma_r(const dzso_params* P, double r);       /* top-hat rms at a = 1 */
/* tables: a[n+1], drift[n], kick1[n], kick2[n], rlc[n+1] (Mpc/h), rlat[n+1] */
void dzso_tables(const dzso_params* P, double* a, double* drift, double* kick1,
                 double* kick2, double* rlc, uint64_t* rlat);

/* ---- FFT (fft.c): unnormalised, sign -1 forward, +1 backward ---- */
void dzso_fft1(int n, double* re_im, int sign);
void dzso_fft3(int n0, int n1, int n2, double* re_im, int sign);

/* ---- initial conditions (ics.c) ---- */
/* c-th output (c >= 0) of the SplitMix64 stream started at state seed */
uint64_t dzso_splitmix64_at(uint64_t seed, uint64_t c);
void dzso_white_noise(uint64_t seed, int n1d, double* w);
void dzso_ics(const dzso_params* P, uint32_t* u, double* p, uint32_t* k,
              uint32_t* id, uint8_t* fl);

/* ---- sort (tree.c) ---- */
uint64_t dzso_morton_key(uint32_t ux, uint32_t uy, uint32_t uz);
void dzso_sort(int64_t n, const uint32_t* u, uint64_t* key_out, int64_t* perm_out);

/* ---- PM (pm.c) ---- */
void dzso_cic_delta(const dzso_params* P, int64_t n, const uint32_t* u,
                    const uint32_t* k, double* delta);
void dzso_pm_potential(const dzso_params* P, const double* delta, double* phi);
void dzso_pm_accel(const dzso_params* P, const double* phi, int64_t n,
                   const uint32_t* u, double* g, const int64_t* sample,
                   int64_t nsample);

/* ---- short-range tree force (tree.c) ----
 * u, k in Morton-sorted order.  If nsample > 0 only the particles listed are
 * evaluated; g of the others is left untouched. */
void dzso_tree_accel(const dzso_params* P, int64_t n, const uint32_t* u,
                     const uint32_t* k, double* g, const int64_t* sample,
                     int64_t nsample);
double dzso_pair_factor(const dzso_params* P, double r, double h);
int64_t dzso_count_groups(const dzso_params* P, int64_t n, const uint32_t* u,
                          int64_t* group_start, int64_t* group_count);
int64_t dzso_interaction_count(const dzso_params* P, int64_t n, const uint32_t* u,
                               const uint32_t* k, int64_t group_index);

/* ---- DZS merge (merge.c) ----
 * In place on Morton-sorted arrays; returns the new particle count.  amin2 is
 * the squared smallest acceleration inside the lightcone (dynamical
 * criterion only; see dzso_amin2). */
int64_t dzso_merge(const dzso_params* P, int64_t n, uint64_t rlat, double amin2, uint32_t* u,
                   double* p, uint32_t* k, uint32_t* id, uint8_t* fl);
/* min over particles not yet crossed of |g|^2 (g [3][n]); +inf if none */
double dzso_amin2(int64_t n, const double* g, const uint8_t* fl);
int32_t dzso_merge_jmin(const dzso_params* P);
uint64_t dzso_merge_threshold(const dzso_params* P, uint64_t rlat, int32_t level);

/* ---- step (step.c) ---- */
/* total acceleration g = PM + tree of the particle set (any order, g in the
 * same order); parts bit 0 = PM, bit 1 = tree */
void dzso_accel(const dzso_params* P, int64_t n, const uint32_t* u,
                const uint32_t* k, double* g, int32_t parts,
                const int64_t* sample, int64_t nsample);
/* opening kick + drift + crossing (state in any order) */
int64_t dzso_kick_drift_cross(const dzso_params* P, int32_t step, int64_t n,
                              uint32_t* u, double* p, const double* g,
                              const uint32_t* k, const uint32_t* id, uint8_t* fl,
                              dzso_record* rec);
/* one full KDK step; arrays sized >= n; returns new n (after merges) or -1.
 * On return the state is Morton-sorted and g holds the new accelerations. */
int64_t dzso_step(const dzso_params* P, int32_t step, int64_t n, uint32_t* u,
                  double* p, double* g, uint32_t* k, uint32_t* id, uint8_t* fl,
                  dzso_record* rec, int64_t* nrec);
/* Sum k, Sum k p[3], Sum k x[3] (Mpc/h), N */
void dzso_diagnostics(const dzso_params* P, int64_t n, const uint32_t* u,
                      const double* p, const uint32_t* k, double out[8]);
/* PHYSICAL mode: flag particles outside R_lc(a_init) as crossed, no record */
void dzso_initial_flags(const dzso_params* P, int64_t n, const uint32_t* u, uint8_t* fl);

/* ---- lightcone observables (observe.c) ---- */
/* RING-ordered pixel of the direction (x, y, z) on the equal-area sphere
 * pixelisation with 12 nside^2 pixels (Górski et al. 2005); (0,0,0) -> +z */
int64_t dzso_ang2pix_ring(int64_t nside, double x, double y, double z);
/* ring index (1 .. 4 nside - 1, north to south), 1-based position j in the
 * ring, and the centre z = cos(theta), phi of a pixel; any pointer may be NULL */
void dzso_pix2ring(int64_t nside, int64_t pix, int64_t* ring, int64_t* j, double* z, double* phi);
void dzso_pix2vec_ring(int64_t nside, int64_t pix, double v[3]);
/* add the mass k of every record with a_lo <= a_cross < a_hi to the pixel of
 * its direction from the observer at the box centre (map: 12 nside^2) */
void dzso_skymap(const dzso_params* P, int64_t nrec, const dzso_record* rec, int64_t nside, double a_lo,
                 double a_hi, uint64_t* map);
/* the same for n points: v [3][n] -> pix [n]; pix [n] -> centres v [3][n] */
void dzso_ang2pix_ring_many(int64_t nside, int64_t n, const double* v, int64_t* pix);
void dzso_pix2vec_ring_many(int64_t nside, int64_t n, const int64_t* pix, double* v);
/* NGP mass of the records with a_lo <= a_cross < a_hi on a mesh^3 grid of the
 * box ([i][j][l], x* / L * mesh floored, clamped to the last cell) */
void dzso_lcdensity(const dzso_params* P, int64_t nrec, const dzso_record* rec, int64_t mesh, double a_lo,
                    double a_hi, uint64_t* grid);
void dzso_pix2zphi_ring_many(int64_t nside, int64_t n, const int64_t* pix, double* z, double* phi);

/* ---- friends-of-friends haloes (fof.c) ---- */
typedef struct {
  int64_t first;   /* smallest member index (labels the halo) */
  int64_t count;   /* particles */
  uint64_t mass;   /* sum k */
  double x[3];     /* centre of mass, Mpc/h, wrapped into [0, L) */
  uint64_t rmax2;  /* largest squared lattice distance of a member from the observer */
} dzso_halo;
/* linking threshold on the squared lattice distance: floor((link 2^32 / n1d)^2) */
uint64_t dzso_fof_threshold(const dzso_params* P, double link);
/* haloes (components with >= nmin particles) of the set u[3][n], masses k;
 * label[i] (may be NULL) = first member of i's halo or -1; returns the halo
 * count, haloes in increasing first-member order (halos sized >= n) */
int64_t dzso_fof(const dzso_params* P, int64_t n, const uint32_t* u, const uint32_t* k, double link, int32_t nmin,
                 int64_t* label, dzso_halo* halos);

#endif
