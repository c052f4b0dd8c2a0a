// ics.cu -- Zel'dovich initial conditions on the GPU (the paper evolves its
// initial conditions with linear theory to z ~ 50, Fig. 1 caption).
//
// White noise on the n^3 particle lattice: SplitMix64 (Steele, Lea & Flood
// 2014) used as a counter-based generator, outputs 2i and 2i+1 of the stream
// started at the seed, Box-Muller.  delta_k = W_k sqrt(n^3 P(k) / L^3) with the
// BBKS transfer function normalised to sigma8; psi_k = i k delta_k / k^2 with
// k = 0 and each axis' Nyquist plane set to zero; x = q + D+ psi on the
// lattice, p = a^2 E f D+ psi.  Always FP64.
#include <cmath>
#include <vector>

#include "common.cuh"

namespace dzs {

template <class R>
std::vector<cplx<R>> twiddles(int n);

namespace {

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t c) {
  uint64_t z = seed + (c + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_noise(uint64_t seed, int64_t n, double* __restrict__ w) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t r0 = splitmix64_at(seed, 2 * (uint64_t)i), r1 = splitmix64_at(seed, 2 * (uint64_t)i + 1);
    double u1 = ((double)(r0 >> 11) + 1.0) * 0x1.0p-53;
    double u2 = (double)(r1 >> 11) * 0x1.0p-53;
    w[i] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
  }
}

struct IcsConst {
  int n1;
  double kf, norm_amp, ns, om_h;
};

__device__ double bbks_shape_dev(double k, double ns, double om_h) {
  double q = k / om_h, t = 1.0;
  if (q > 1e-12) {
    double a = 16.1 * q, b = 5.46 * q, c = 6.71 * q;
    double poly = 1.0 + 3.89 * q + a * a + b * b * b + c * c * c * c;
    t = log(1.0 + 2.34 * q) / (2.34 * q) * pow(poly, -0.25);
  }
  return pow(k, ns) * t * t;
}

__device__ __forceinline__ int signed_index(int m, int n) { return m <= n / 2 ? m : m - n; }

// delta_k = W_k sqrt(n^3 A shape(k) / L^3), in place on the half spectrum
__global__ void k_ics_delta(cplx<double>* __restrict__ s, IcsConst C) {
  const int n = C.n1, hn = n / 2 + 1;
  const int64_t total = (int64_t)n * n * hn;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int kz = (int)(t % hn), iy = (int)((t / hn) % n), ix = (int)(t / ((int64_t)hn * n));
    double nx = signed_index(ix, n), ny = signed_index(iy, n), nz = kz;
    double k = C.kf * sqrt(nx * nx + ny * ny + nz * nz);
    double f = k > 0.0 ? sqrt(C.norm_amp * bbks_shape_dev(k, C.ns, C.om_h)) : 0.0;
    s[t].x *= f;
    s[t].y *= f;
  }
}

// psi component ax: i k_ax delta_k / k^2, Nyquist plane of axis ax zeroed
__global__ void k_ics_psi(const cplx<double>* __restrict__ d, cplx<double>* __restrict__ o, IcsConst C, int ax) {
  const int n = C.n1, hn = n / 2 + 1;
  const int64_t total = (int64_t)n * n * hn;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int kz = (int)(t % hn), iy = (int)((t / hn) % n), ix = (int)(t / ((int64_t)hn * n));
    int m[3] = {ix, iy, kz};
    double nv[3] = {(double)signed_index(ix, n), (double)signed_index(iy, n), (double)kz};
    double k2 = C.kf * C.kf * (nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
    cplx<double> v = {0.0, 0.0};
    bool nyq = (n % 2 == 0) && (m[ax] == n / 2);
    if (k2 > 0.0 && !nyq) {
      double kc = C.kf * nv[ax] / k2;
      v = {-kc * d[t].y, kc * d[t].x};
    }
    o[t] = v;
  }
}

template <class R>
__global__ void k_ics_place(const double* __restrict__ psi, int ax, int n1, int64_t cap, double dlat, double pfac,
                            double inv_n3, uint32_t* __restrict__ u, R* __restrict__ p) {
  const int64_t n = (int64_t)n1 * n1 * n1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int mv[3] = {(int)(i / ((int64_t)n1 * n1)), (int)((i / n1) % n1), (int)(i % n1)};
    double ps = psi[i] * inv_n3;
    uint64_t q = ((uint64_t)mv[ax] << 32) / (uint64_t)n1;
    long long du = __double2ll_rn(dlat * ps);
    u[ax * cap + i] = (uint32_t)(q + (uint64_t)du);
    p[ax * cap + i] = (R)(pfac * ps);
  }
}

__global__ void k_ics_finish(int64_t n, int64_t cap, const uint32_t* __restrict__ u, uint32_t* __restrict__ k,
                             uint32_t* __restrict__ id, uint8_t* __restrict__ fl, uint64_t r20,
                             int32_t* __restrict__ d_n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    k[i] = 1;
    id[i] = (uint32_t)i;
    fl[i] = dist2_obs(u[i], u[cap + i], u[2 * cap + i]) >= r20 ? kFlCrossed : 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *d_n = (int32_t)n;
}

}  // namespace

void launch_ics(dzs_ctx* c) {
  const int n1 = c->n1;
  const int64_t n = c->N0, hn = n1 / 2 + 1;
  const int64_t nspec = (int64_t)n1 * n1 * hn;
  // scratch from the arena (no allocation, so no device-wide synchronisation
  // while other contexts run): the noise / displacement grid and the IC
  // twiddles in the conversion scratch (24 N0 bytes), the two half spectra
  // (16 n1^2 (n1/2 + 1) <= 12 N0 bytes each for n1 >= 4) in g and gsave,
  // which the first force evaluation overwrites
  double* w = (double*)c->B.convert;
  cplx<double>* tw = (cplx<double>*)(w + n);
  cplx<double>* sd = (cplx<double>*)c->B.g;
  cplx<double>* sw = (cplx<double>*)c->B.gsave;
  auto twh = twiddles<double>(n1);
  cudaMemcpyAsync(tw, twh.data(), sizeof(cplx<double>) * twh.size(), cudaMemcpyHostToDevice, c->stream);
  k_noise<<<grid_for(n), kThreads, 0, c->stream>>>(c->P.seed, n, w);
  fft_r2c_3d<double>(c, w, sd, n1, tw);
  IcsConst C;
  C.n1 = n1;
  C.kf = 2.0 * M_PI / c->P.box;
  C.norm_amp = (double)n / (c->P.box * c->P.box * c->P.box) * c->T.power_amp;
  C.ns = c->P.ns;
  C.om_h = c->P.omega_m * c->P.hubble;
  k_ics_delta<<<grid_for(nspec), kThreads, 0, c->stream>>>(sd, C);
  double ai = c->T.a[0];
  double pfac = ai * ai * c->T.e_i * c->T.f_i * c->T.dplus_i;
  double dlat = c->T.dplus_i * c->lat;
  for (int ax = 0; ax < 3; ++ax) {
    k_ics_psi<<<grid_for(nspec), kThreads, 0, c->stream>>>(sd, sw, C, ax);
    fft_c2r_3d<double>(c, sw, w, n1, tw, nullptr, 0.0);
    if (c->fp64)
      k_ics_place<double><<<grid_for(n), kThreads, 0, c->stream>>>(w, ax, n1, c->cap, dlat, pfac, 1.0 / (double)n,
                                                                   c->B.u, (double*)c->B.p);
    else
      k_ics_place<float><<<grid_for(n), kThreads, 0, c->stream>>>(w, ax, n1, c->cap, dlat, pfac, 1.0 / (double)n,
                                                                  c->B.u, (float*)c->B.p);
  }
  uint64_t r0 = c->T.rlat[0];
  k_ics_finish<<<grid_for(n), kThreads, 0, c->stream>>>(n, c->cap, c->B.u, c->B.k, c->B.id, c->B.fl, r0 * r0, c->B.n);
}

}  // namespace dzs
