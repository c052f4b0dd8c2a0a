/*
 * cosmo.c -- oracle: FP64 background cosmology and the per-step time tables.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper fixes the lightcone radius as the comoving distance travelled by
 * light (Sec. 1, footnote on R_lc; Fig. 1) and integrates particles with
 * global steps (Sec. 2.1).  The integrals themselves are not printed; they are
 * the textbook ones for a matter + Lambda universe with H0 = 1:
 *   E(a)   = sqrt(Om a^-3 + Ok a^-2 + OL)
 *   drift  = int da / (a^3 E)        (dx = p dt / a^2, dt = da / (a E))
 *   kick   = int da / (a^2 E)        (dp = -grad(phi) dt / a)
 *   chi(a) = c/H0 int_a^1 da / (a^2 E)
 *   D+(a)  proportional to E(a) int_0^a da' / (a' E)^3, D+(1) = 1
 * Each integral is evaluated by adaptive Simpson quadrature to ~1e-15.
 */
#include <math.h>

#include "oracle.h"

#define C_OVER_H0 2997.92458 /* Mpc/h */

typedef double (*integrand_fn)(const dzso_params*, double);

static double simpson_rec(integrand_fn f, const dzso_params* P, double a, double b,
                          double fa, double fm, double fb, double whole, double tol_abs,
                          int depth) {
  double m = 0.5 * (a + b);
  double lm = 0.5 * (a + m), rm = 0.5 * (m + b);
  double flm = f(P, lm), frm = f(P, rm);
  double left = (m - a) / 6.0 * (fa + 4.0 * flm + fm);
  double right = (b - m) / 6.0 * (fm + 4.0 * frm + fb);
  double both = left + right;
  /* stop at relative 1e-15 of this piece or at its share of the absolute
   * tolerance; the returned value is Richardson-extrapolated */
  double tol = 1e-15 * fabs(both);
  if (tol < tol_abs) tol = tol_abs;
  if (depth <= 0 || fabs(both - whole) <= 15.0 * tol) return both + (both - whole) / 15.0;
  return simpson_rec(f, P, a, m, fa, flm, fm, left, 0.5 * tol_abs, depth - 1) +
         simpson_rec(f, P, m, b, fm, frm, fb, right, 0.5 * tol_abs, depth - 1);
}

/* integral of f over [a, b]: a 256-panel Simpson estimate fixes the absolute
 * tolerance (1e-15 of the total), then each panel is refined adaptively */
static double integrate(integrand_fn f, const dzso_params* P, double a, double b) {
  if (a == b) return 0.0;
  enum { panels = 256 };
  double x[panels + 1], fx[panels + 1], fm[panels], whole[panels];
  double rough = 0.0;
  for (int i = 0; i <= panels; ++i) {
    x[i] = (i == panels) ? b : a + (b - a) * i / panels;
    fx[i] = f(P, x[i]);
  }
  for (int i = 0; i < panels; ++i) {
    fm[i] = f(P, 0.5 * (x[i] + x[i + 1]));
    whole[i] = (x[i + 1] - x[i]) / 6.0 * (fx[i] + 4.0 * fm[i] + fx[i + 1]);
    rough += whole[i];
  }
  double tol_abs = 1e-15 * fabs(rough) / panels;
  double sum = 0.0;
  for (int i = 0; i < panels; ++i)
    sum += simpson_rec(f, P, x[i], x[i + 1], fx[i], fm[i], fx[i + 1], whole[i], tol_abs, 30);
  return sum;
}

double dzso_hubble_e(const dzso_params* P, double a) {
  double ok = 1.0 - P->omega_m - P->omega_l;
  return sqrt(P->omega_m / (a * a * a) + ok / (a * a) + P->omega_l);
}

static double f_drift(const dzso_params* P, double a) {
  return 1.0 / (a * a * a * dzso_hubble_e(P, a));
}
static double f_kick(const dzso_params* P, double a) {
  return 1.0 / (a * a * dzso_hubble_e(P, a));
}
/* growth integrand after a = t^2 (removes the a^(1/2) behaviour at a -> 0):
 * int_0^a da / (a E)^3 = int_0^sqrt(a) 2 t dt / (t^2 E(t^2))^3 */
static double f_growth(const dzso_params* P, double t) {
  if (t == 0.0) {
    /* (aE)^3 -> Om^1.5 a^-1.5 as a -> 0, so 2t/(aE)^3 -> 0 */
    return 0.0;
  }
  double a = t * t;
  double ae = a * dzso_hubble_e(P, a);
  return 2.0 * t / (ae * ae * ae);
}

double dzso_drift_factor(const dzso_params* P, double a0, double a1) {
  return integrate(f_drift, P, a0, a1);
}
double dzso_kick_factor(const dzso_params* P, double a0, double a1) {
  return integrate(f_kick, P, a0, a1);
}
double dzso_chi(const dzso_params* P, double a) {
  return C_OVER_H0 * integrate(f_kick, P, a, 1.0);
}

static double growth_unnorm(const dzso_params* P, double a) {
  return dzso_hubble_e(P, a) * integrate(f_growth, P, 0.0, sqrt(a));
}

double dzso_growth(const dzso_params* P, double a) {
  return growth_unnorm(P, a) / growth_unnorm(P, 1.0);
}

/* f = dlnD/dlna = a E'/E + 1 / (a^2 E^3 I(a)), I = int_0^a da/(aE)^3,
 * E' = dE/da = -(3 Om a^-4 + 2 Ok a^-3) / (2 E) */
double dzso_growth_rate(const dzso_params* P, double a) {
  double e = dzso_hubble_e(P, a);
  double ok = 1.0 - P->omega_m - P->omega_l;
  double de = -(3.0 * P->omega_m / (a * a * a * a) + 2.0 * ok / (a * a * a)) / (2.0 * e);
  double I = integrate(f_growth, P, 0.0, sqrt(a));
  return a * de / e + 1.0 / (a * a * e * e * e * I);
}

/* ---- linear power spectrum: P(k) = A k^ns T_BBKS(q)^2, q = k / (Om h)
 * (Bardeen, Bond, Kaiser & Szalay 1986 transfer function), A from sigma8 ---- */
static double bbks(const dzso_params* P, double k) {
  double q = k / (P->omega_m * P->hubble);
  if (q < 1e-12) return 1.0;
  double t1 = log(1.0 + 2.34 * q) / (2.34 * q);
  double poly = 1.0 + 3.89 * q + pow(16.1 * q, 2) + pow(5.46 * q, 3) + pow(6.71 * q, 4);
  return t1 * pow(poly, -0.25);
}

static double tophat_w(double x) {
  if (x < 1e-3) return 1.0 - x * x / 10.0 + x * x * x * x / 280.0;
  return 3.0 * (sin(x) - x * cos(x)) / (x * x * x);
}

/* filter radius of the sigma integral in progress; the oracle evaluates the
 * spectrum normalisation single-threaded */
static double g_radius;

/* d sigma^2 / d ln k for the un-normalised spectrum */
static double f_sigma(const dzso_params* P, double lnk) {
  double k = exp(lnk);
  double t = bbks(P, k);
  double w = tophat_w(k * g_radius);
  return k * k * k * pow(k, P->ns) * t * t * w * w / (2.0 * M_PI * M_PI);
}

static double sigma2_unnorm(const dzso_params* P, double r) {
  g_radius = r;
  return integrate(f_sigma, P, log(1e-7), log(1e4));
}

double dzso_power_amplitude(const dzso_params* P) {
  return P->sigma8 * P->sigma8 / sigma2_unnorm(P, 8.0);
}

double dzso_power_shape(const dzso_params* P, double k) {
  if (k <= 0.0) return 0.0;
  double t = bbks(P, k);
  return pow(k, P->ns) * t * t;
}

double dzso_power(const dzso_params* P, double k) {
  return dzso_power_amplitude(P) * dzso_power_shape(P, k);
}

double dzso_sigma_r(const dzso_params* P, double r) {
  return sqrt(dzso_power_amplitude(P) * sigma2_unnorm(P, r));
}

/* ---- per-step tables: a_n = exp(ln a_i + n dlna), dlna = -ln a_i / nsteps,
 * half steps at the ln-a midpoint; a_N = 1 exactly.
 * R_lc: SWEEP    R(a) = (sqrt(3) L / 2) chi(a) / chi(a_i)
 *       PHYSICAL R(a) = min(chi(a), sqrt(3) L / 2)
 * rlat_n = floor(R(a_n) / L * 2^32). ---- */
void dzso_tables(const dzso_params* P, double* a, double* drift, double* kick1,
                 double* kick2, double* rlc, uint64_t* rlat) {
  int ns = P->nsteps;
  double lnai = -log1p(P->z_init);
  double dlna = -lnai / ns;
  for (int n = 0; n <= ns; ++n) a[n] = (n == ns) ? 1.0 : exp(lnai + n * dlna);
  for (int n = 0; n < ns; ++n) {
    double ah = exp(lnai + (n + 0.5) * dlna);
    drift[n] = dzso_drift_factor(P, a[n], a[n + 1]);
    kick1[n] = dzso_kick_factor(P, a[n], ah);
    kick2[n] = dzso_kick_factor(P, ah, a[n + 1]);
  }
  double rmax = sqrt(3.0) * P->box / 2.0;
  double chi0 = dzso_chi(P, a[0]);
  for (int n = 0; n <= ns; ++n) {
    double chi = dzso_chi(P, a[n]);
    double r;
    if (P->rlc_mode == DZSO_RLC_SWEEP)
      r = rmax * chi / chi0;
    else
      r = chi < rmax ? chi : rmax;
    rlc[n] = r;
    rlat[n] = (uint64_t)floor(r / P->box * 4294967296.0);
  }
}
