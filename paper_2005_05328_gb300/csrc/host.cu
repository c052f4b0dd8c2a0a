// host.cu -- FP64 host tables of the DZS step: background expansion, the
// drift/kick time integrals of the global KDK steps, the lightcone radius
// R_lc(a) and the linear-theory quantities used by the initial conditions.
//
// Paper: R_lc is the comoving distance light travels (Sec. 1 footnote, Fig. 1);
// particles advance on global steps (Sec. 2.1).  With H0 = 1 and p = a^2 dx/dt:
//   drift D(a0, a1) = int da / (a^3 E) = int dln a / (a^2 E)
//   kick  K(a0, a1) = int da / (a^2 E) = int dln a / (a E)
//   chi(a) = c/H0 int_a^1 dln a / (a E)
//   D+(a) ~ E(a) int_0^a da / (a E)^3, f = dln D+ / dln a.
// All integrals use composite Gauss-Legendre quadrature in ln a.
#include <cmath>
#include <vector>

#include "common.cuh"

namespace dzs {
namespace {

constexpr double kCOverH0 = 2997.92458;  // Mpc/h
constexpr int kGL = 20;

struct GaussLegendre {
  double x[kGL], w[kGL];
  GaussLegendre() {
    // roots of P_n by Newton iteration from the Chebyshev-like guess
    const int n = kGL;
    for (int i = 0; i < n; ++i) {
      double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
          double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = pk;
        }
        double dp = n * (z * p1 - p0) / (z * z - 1.0);
        double dz = p1 / dp;
        z -= dz;
        if (std::fabs(dz) < 1e-16) break;
      }
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      double dp = n * (z * p1 - p0) / (z * z - 1.0);
      x[i] = z;
      w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
  }
};

const GaussLegendre& gl() {
  static GaussLegendre g;
  return g;
}

template <class F>
double quad(F f, double lo, double hi, int panels) {
  if (lo == hi) return 0.0;
  const GaussLegendre& g = gl();
  double h = (hi - lo) / panels, sum = 0.0;
  for (int p = 0; p < panels; ++p) {
    double a = lo + p * h, mid = a + 0.5 * h, part = 0.0;
    for (int i = 0; i < kGL; ++i) part += g.w[i] * f(mid + 0.5 * h * g.x[i]);
    sum += 0.5 * h * part;
  }
  return sum;
}

struct Cosmo {
  double om, ol, ok;
  explicit Cosmo(const dzs_params& P) : om(P.omega_m), ol(P.omega_l), ok(1.0 - P.omega_m - P.omega_l) {}
  double E(double a) const { return std::sqrt(om / (a * a * a) + ok / (a * a) + ol); }
  double drift(double a0, double a1) const {
    return quad([&](double s) { double a = std::exp(s); return 1.0 / (a * a * E(a)); },
                std::log(a0), std::log(a1), 8);
  }
  double kick(double a0, double a1) const {
    return quad([&](double s) { double a = std::exp(s); return 1.0 / (a * E(a)); },
                std::log(a0), std::log(a1), 8);
  }
  double chi(double a) const {
    return kCOverH0 * quad([&](double s) { double a1 = std::exp(s); return 1.0 / (a1 * E(a1)); },
                           std::log(a), 0.0, 256);
  }
  // int_0^a da / (a E)^3 in ln a from a = 1e-9 (the integrand ~ a^2.5 below)
  double growth_integral(double a) const {
    return quad([&](double s) { double x = std::exp(s); double ae = x * E(x); return x / (ae * ae * ae); },
                std::log(1e-9), std::log(a), 256);
  }
  double growth(double a) const { return E(a) * growth_integral(a) / (E(1.0) * growth_integral(1.0)); }
  double growth_rate(double a) const {
    double e = E(a);
    double de = -(3.0 * om / (a * a * a * a) + 2.0 * ok / (a * a * a)) / (2.0 * e);
    return a * de / e + 1.0 / (a * a * e * e * e * growth_integral(a));
  }
};

double tophat(double x) {
  if (x < 1e-3) return 1.0 - x * x / 10.0;
  return 3.0 * (std::sin(x) - x * std::cos(x)) / (x * x * x);
}

}  // namespace

// k^ns T_BBKS(k / (Om h))^2 (Bardeen, Bond, Kaiser & Szalay 1986)
double bbks_shape(const dzs_params& P, double k) {
  if (k <= 0.0) return 0.0;
  double q = k / (P.omega_m * P.hubble);
  double t = 1.0;
  if (q > 1e-12) {
    double poly = 1.0 + 3.89 * q + (16.1 * q) * (16.1 * q) + std::pow(5.46 * q, 3) + std::pow(6.71 * q, 4);
    t = std::log(1.0 + 2.34 * q) / (2.34 * q) * std::pow(poly, -0.25);
  }
  return std::pow(k, P.ns) * t * t;
}

void compute_tables(const dzs_params& P, Tables& T) {
  Cosmo cm(P);
  int ns = P.nsteps;
  double lnai = -std::log1p(P.z_init), dl = -lnai / ns;
  T.a.assign(ns + 1, 0.0);
  T.drift.assign(ns, 0.0);
  T.kick1.assign(ns, 0.0);
  T.kick2.assign(ns, 0.0);
  T.rlc.assign(ns + 1, 0.0);
  T.rlat.assign(ns + 1, 0);
  for (int n = 0; n <= ns; ++n) T.a[n] = (n == ns) ? 1.0 : std::exp(lnai + n * dl);
  for (int n = 0; n < ns; ++n) {
    double ah = std::exp(lnai + (n + 0.5) * dl);
    T.drift[n] = cm.drift(T.a[n], T.a[n + 1]);
    T.kick1[n] = cm.kick(T.a[n], ah);
    T.kick2[n] = cm.kick(ah, T.a[n + 1]);
  }
  double rmax = std::sqrt(3.0) * P.box / 2.0;
  double chi0 = cm.chi(T.a[0]);
  for (int n = 0; n <= ns; ++n) {
    double chi = cm.chi(T.a[n]);
    double r = (P.rlc_mode == DZS_RLC_SWEEP) ? rmax * chi / chi0 : std::fmin(chi, rmax);
    T.rlc[n] = r;
    T.rlat[n] = (uint64_t)std::floor(r / P.box * 4294967296.0);
  }
  double ai = T.a[0];
  T.dplus_i = cm.growth(ai);
  T.f_i = cm.growth_rate(ai);
  T.e_i = cm.E(ai);
  // sigma^2(8 Mpc/h) of the unnormalised spectrum, in ln k
  double s2 = quad([&](double s) {
                     double k = std::exp(s), w = tophat(8.0 * k);
                     return k * k * k * bbks_shape(P, k) * w * w / (2.0 * M_PI * M_PI);
                   },
                   std::log(1e-7), std::log(1e4), 2048);
  T.power_amp = P.sigma8 * P.sigma8 / s2;
}

int sm_count() {
  static int cache[256] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return 1;
  if (cache[dev] <= 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 1;
    cache[dev] = n;
  }
  return cache[dev];
}

}  // namespace dzs
