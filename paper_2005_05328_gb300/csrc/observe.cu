// observe.cu -- lightcone observables on the GPU (paper Sec. 3.1.2: sky map
// of the lightcone mass and its angular power spectrum, Fig. 4; Sec. 3.1.3:
// the 3D lightcone, Fig. 5).
//
// Binning: each lightcone record adds its mass k to the RING pixel of its
// direction from the observer and to the NGP cell of its crossing position
// (integer atomics: the maps are exact and independent of the order).  The
// step's record kernel does this as it writes the record; k_observe_records
// does it for records supplied by the caller.
//
// Harmonic analysis of the sky map, a_lm = Omega sum_p map_p conj(Y_lm(p)),
// in the two factors the iso-latitude rings allow:
//   1. per ring r: F_r(m) = sum_j map_j e^{-i m phi_j}   (k_ring_dft)
//   2. per m:      a_lm = Omega sum_r lambda_lm(z_r) F_r(m)   (k_legendre)
// with lambda_lm the orthonormal associated Legendre functions (Condon-
// Shortley phase), advanced in l by the three-term recursion
//   lambda_mm     = -sqrt((2m+1)/(2m)) sqrt(1 - z^2) lambda_{m-1,m-1},
//                   lambda_00 = 1 / sqrt(4 pi)
//   lambda_m+1,m  = z sqrt(2m+3) lambda_mm
//   lambda_lm     = A_lm z lambda_l-1,m - B_lm lambda_l-2,m,
//   A_lm = sqrt((4l^2 - 1) / (l^2 - m^2)),
//   B_lm = sqrt((2l+1)((l-1)^2 - m^2) / ((2l-3)(l^2 - m^2))).
// C_l = (|a_l0|^2 + 2 sum_m>0 |a_lm|^2) / (2l + 1).  Every sum runs in a fixed
// order, so the spectrum is deterministic.
#include <cmath>

#include "common.cuh"
#include "observe.cuh"

namespace dzs {
namespace {

__global__ void k_observe_records(const dzs_lc_record* __restrict__ rec, int64_t n, ObserveTarget o) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const dzs_lc_record r = rec[i];
    observe_record(o, r.k, r.a_cross, r.x);
  }
}

struct RingGeom {
  int64_t nphi, start;
  double z;
  int twof;  // 2 f: the centre of pixel j (0-based) sits at (j + 1 - f) 2 pi / nphi
};

// ring r = 1 .. 4 nside - 1, north to south
__device__ __forceinline__ RingGeom ring_geom(int64_t nside, int64_t r) {
  RingGeom g;
  const double n2 = 3.0 * (double)nside * (double)nside;
  if (r < nside) {
    g.nphi = 4 * r;
    g.start = 2 * r * (r - 1);
    g.z = 1.0 - (double)(r * r) / n2;
    g.twof = 1;
  } else if (r <= 3 * nside) {
    g.nphi = 4 * nside;
    g.start = 2 * nside * (nside - 1) + (r - nside) * 4 * nside;
    g.z = (double)(2 * nside - r) * 2.0 / (3.0 * (double)nside);
    g.twof = ((r + nside) & 1) ? 2 : 1;
  } else {
    const int64_t s = 4 * nside - r;
    g.nphi = 4 * s;
    g.start = 12 * nside * nside - 2 * s * (s + 1);
    g.z = -1.0 + (double)(s * s) / n2;
    g.twof = 1;
  }
  return g;
}

constexpr int kAnchor = 32;  // the phasor is recomputed exactly every kAnchor pixels

// F[r-1][m] for m = 0..lmax; one block per ring, the ring staged in shared memory
__global__ void k_ring_dft(const unsigned long long* __restrict__ map, int64_t nside, int lmax,
                           double2* __restrict__ F) {
  extern __shared__ double ring[];
  const int64_t r = blockIdx.x + 1;
  const RingGeom g = ring_geom(nside, r);
  for (int64_t j = threadIdx.x; j < g.nphi; j += blockDim.x) ring[j] = (double)map[g.start + j];
  __syncthreads();
  const int64_t per = 2 * g.nphi;  // angles are pi q / nphi with q taken mod 2 nphi
  for (int m = threadIdx.x; m <= lmax; m += blockDim.x) {
    double sst, cst;
    sincospi((double)((2 * (int64_t)m) % per) / (double)g.nphi, &sst, &cst);
    double re = 0.0, im = 0.0;
    for (int64_t j0 = 0; j0 < g.nphi; j0 += kAnchor) {
      const int64_t q = ((int64_t)m * (2 * j0 + 2 - g.twof)) % per;
      double s, c;
      sincospi((double)q / (double)g.nphi, &s, &c);
      const int64_t j1 = j0 + kAnchor < g.nphi ? j0 + kAnchor : g.nphi;
      for (int64_t j = j0; j < j1; ++j) {
        const double v = ring[j];
        re += v * c;
        im -= v * s;
        const double c2 = c * cst - s * sst;
        s = s * cst + c * sst;
        c = c2;
      }
    }
    F[(r - 1) * (lmax + 1) + m] = make_double2(re, im);
  }
}

constexpr int kLegThreads = 256;
constexpr int kLegWarps = kLegThreads / 32;
constexpr int kRingsPerThread = 4;
constexpr int kLTile = 64;

__host__ __device__ inline int64_t alm_index(int lmax, int l, int m) {
  return (int64_t)m * (2 * lmax + 1 - m) / 2 + l;
}

// one block per m: alm[l, m] += Omega sum over rings, ring chunks in order
__global__ void __launch_bounds__(kLegThreads) k_legendre(const double2* __restrict__ F, int64_t nside, int lmax,
                                                          double omega, double2* __restrict__ alm) {
  extern __shared__ double sh[];
  double* A = sh;                                   // [lmax + 1]
  double* Bc = A + (lmax + 1);                      // [lmax + 1]
  double2* part = (double2*)(Bc + (lmax + 1));      // [kLegWarps][kLTile]
  const int m = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int l = m + 2 + threadIdx.x; l <= lmax; l += blockDim.x) {
    const double dl = l, dm = m, d = dl * dl - dm * dm;
    A[l] = sqrt((4.0 * dl * dl - 1.0) / d);
    Bc[l] = sqrt((2.0 * dl + 1.0) * ((dl - 1.0) * (dl - 1.0) - dm * dm) / ((2.0 * dl - 3.0) * d));
  }
  const int64_t nrings = 4 * nside - 1;
  const int64_t chunk = (int64_t)kLegThreads * kRingsPerThread;
  for (int64_t c0 = 0; c0 < nrings; c0 += chunk) {
    double z[kRingsPerThread], l1[kRingsPerThread], l2[kRingsPerThread];
    double2 f[kRingsPerThread];
#pragma unroll
    for (int q = 0; q < kRingsPerThread; ++q) {
      const int64_t r = c0 + threadIdx.x + (int64_t)q * kLegThreads;  // 0-based ring
      if (r < nrings) {
        z[q] = ring_geom(nside, r + 1).z;
        f[q] = F[r * (lmax + 1) + m];
        // lambda_mm by the stable product
        const double s = sqrt((1.0 - z[q]) * (1.0 + z[q]));
        double v = 0.28209479177387814;  // 1 / sqrt(4 pi)
        for (int k = 1; k <= m; ++k) v *= -sqrt((2.0 * k + 1.0) / (2.0 * k)) * s;
        l2[q] = 0.0;
        l1[q] = v;
      } else {
        z[q] = 0.0;
        f[q] = make_double2(0.0, 0.0);
        l1[q] = l2[q] = 0.0;
      }
    }
    __syncthreads();  // A, B ready (first chunk); part free (later chunks)
    for (int lt = m; lt <= lmax; lt += kLTile) {
      const int lend = lt + kLTile - 1 < lmax ? lt + kLTile - 1 : lmax;
      for (int l = lt; l <= lend; ++l) {
        double re = 0.0, im = 0.0;
#pragma unroll
        for (int q = 0; q < kRingsPerThread; ++q) {
          double lam;
          if (l == m) {
            lam = l1[q];
          } else if (l == m + 1) {
            lam = z[q] * sqrt(2.0 * m + 3.0) * l1[q];
            l2[q] = l1[q];
            l1[q] = lam;
          } else {
            lam = A[l] * z[q] * l1[q] - Bc[l] * l2[q];
            l2[q] = l1[q];
            l1[q] = lam;
          }
          re += lam * f[q].x;
          im += lam * f[q].y;
        }
        for (int o = 16; o > 0; o >>= 1) {
          re += __shfl_down_sync(0xffffffffu, re, o);
          im += __shfl_down_sync(0xffffffffu, im, o);
        }
        if (lane == 0) part[w * kLTile + (l - lt)] = make_double2(re, im);
      }
      __syncthreads();
      if (threadIdx.x < kLTile && lt + (int)threadIdx.x <= lend) {
        double2 s = make_double2(0.0, 0.0);
        for (int q = 0; q < kLegWarps; ++q) {
          s.x += part[q * kLTile + threadIdx.x].x;
          s.y += part[q * kLTile + threadIdx.x].y;
        }
        double2* out = &alm[alm_index(lmax, lt + threadIdx.x, m)];
        double2 acc = c0 == 0 ? make_double2(0.0, 0.0) : *out;
        acc.x += omega * s.x;
        acc.y += omega * s.y;
        *out = acc;
      }
      __syncthreads();
    }
  }
}

__global__ void k_cl(const double2* __restrict__ alm, int lmax, double* __restrict__ cl) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l > lmax) return;
  double s = 0.0;
  for (int m = 0; m <= l; ++m) {
    const double2 a = alm[alm_index(lmax, l, m)];
    const double p = a.x * a.x + a.y * a.y;
    s += m == 0 ? p : 2.0 * p;
  }
  cl[l] = s / (2.0 * l + 1.0);
}

}  // namespace

void launch_observe_records(dzs_ctx* c, const dzs_lc_record* d_rec, int64_t n) {
  if (n <= 0) return;
  c->launches += 1;
  k_observe_records<<<grid_for(n), kThreads, 0, c->stream>>>(d_rec, n, c->obs);
}

size_t sht_work_bytes(int64_t nside, int lmax) {
  const size_t nr = (size_t)(4 * nside - 1), nl = (size_t)lmax + 1;
  const size_t nalm = nl * (nl + 1) / 2;
  return 16 * nr * nl + 16 * nalm + 8 * nl + 256;
}

size_t sht_shared_bytes(int lmax) { return 16 * ((size_t)lmax + 1) + 16 * kLegWarps * kLTile; }

// a_lm (m-major, index m (2 lmax + 1 - m) / 2 + l, complex interleaved) and C_l
// of the context's sky map into work: [F | alm | cl]
void launch_sht(dzs_ctx* c, int lmax, void* work, double2** d_alm, double** d_cl) {
  const int64_t nside = c->obs.nside, nr = 4 * nside - 1;
  char* w = (char*)work;
  double2* F = (double2*)w;
  double2* alm = (double2*)(w + 16 * (size_t)nr * (lmax + 1));
  const size_t nalm = (size_t)(lmax + 1) * (lmax + 2) / 2;
  double* cl = (double*)((char*)alm + 16 * nalm);
  c->launches += 3;
  const int dft_threads = 256;
  cudaFuncSetAttribute(k_ring_dft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(8 * 4 * nside));
  cudaFuncSetAttribute(k_legendre, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sht_shared_bytes(lmax));
  k_ring_dft<<<(unsigned)nr, dft_threads, 8 * 4 * nside, c->stream>>>(c->obs.sky, nside, lmax, F);
  const double omega = 4.0 * M_PI / (double)(12 * nside * nside);
  k_legendre<<<lmax + 1, kLegThreads, sht_shared_bytes(lmax), c->stream>>>(F, nside, lmax, omega, alm);
  k_cl<<<(lmax + 256) / 256, 256, 0, c->stream>>>(alm, lmax, cl);
  *d_alm = alm;
  *d_cl = cl;
}

// ---- twin-particle displacements (paper Sec. 3.2, integration accuracy):
// particles inside the lightcone (not crossed) in both runs of a twin pair,
// matched by id, the minimum-image distance of their positions over
// h = L / N^(1/3) / 40, binned by the caller's edges.  FP64 with correctly
// rounded operations in a fixed order (the CPU check does the same), integer
// atomics for the counts: exact and independent of the order.

__global__ void k_twin_map(const int32_t* __restrict__ d_n, const uint32_t* __restrict__ id,
                           const uint8_t* __restrict__ fl, int32_t* __restrict__ map, int64_t n0) {
  const int64_t n = *d_n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (fl[i] & kFlCrossed) continue;
    const uint32_t q = id[i];
    if ((int64_t)q < n0) map[q] = (int32_t)i;
  }
}

__global__ void k_twin_disp(const int32_t* __restrict__ d_n, int64_t cap, const uint32_t* __restrict__ u,
                            const uint32_t* __restrict__ id, const uint8_t* __restrict__ fl,
                            const int32_t* __restrict__ map, int64_t capb, const uint32_t* __restrict__ ub,
                            const double* __restrict__ edges, int nbins, double scale, double h, int64_t n0,
                            unsigned long long* __restrict__ counts, unsigned long long* __restrict__ stats) {
  const int64_t n = *d_n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (fl[i] & kFlCrossed) continue;
    const uint32_t q = id[i];
    if ((int64_t)q >= n0) continue;
    const int32_t j = map[q];
    if (j < 0) continue;
    double s = 0.0;
    for (int ax = 0; ax < 3; ++ax) {
      const double d = __dmul_rn((double)(int32_t)(u[ax * cap + i] - ub[ax * capb + j]), scale);
      s = __dadd_rn(s, __dmul_rn(d, d));
    }
    const double ratio = __ddiv_rn(__dsqrt_rn(s), h);
    // bin k: edges[k] <= ratio < edges[k + 1]
    int lo = 0, hi = nbins + 1;  // first edge > ratio, in [lo, hi)
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (edges[mid] <= ratio)
        lo = mid + 1;
      else
        hi = mid;
    }
    const int k = lo - 1;
    if (k >= 0 && k < nbins) atomicAdd(&counts[k], 1ull);
    atomicAdd(&stats[0], 1ull);
    atomicMax(&stats[1], (unsigned long long)__double_as_longlong(ratio));  // ratio >= 0: bits order like values
  }
}

void launch_twin_displacement(dzs_ctx* a, dzs_ctx* b, int32_t* map, const double* edges, int nbins, double h,
                              unsigned long long* counts, unsigned long long* stats) {
  a->launches += 2;
  cudaMemsetAsync(map, 0xff, sizeof(int32_t) * a->N0, a->stream);
  k_twin_map<<<grid_for(b->cap), kThreads, 0, a->stream>>>(b->B.n, b->B.id, b->B.fl, map, a->N0);
  k_twin_disp<<<grid_for(a->cap), kThreads, 0, a->stream>>>(a->B.n, a->cap, a->B.u, a->B.id, a->B.fl, map, b->cap,
                                                             b->B.u, edges, nbins, a->scale, h, a->N0, counts,
                                                             stats);
}

}  // namespace dzs
