// pm.cu -- particle-mesh long-range force (paper Sec. 2.1): atomic-free CIC
// deposit, FFT Poisson solve with the Gaussian split (fft.cu), four-point
// gradient and CIC interpolation back to the particles.
//
// Deposit: the particles are Morton-sorted, so the particles of one mesh cell
// (for M = 2^m the depth-m Morton prefix) are one contiguous run.  A CSR-like
// table start[c] (Morton cell index) is written once per cell by the particle
// that opens each run (covering the empty cells before it), then every mesh
// node gathers k w from the 8 cells it touches.  No atomics: each node sums
// in a fixed order (cell offset, then particle order), so the mesh is
// deterministic.  Mesh node (ix, iy, iz) sits at (ix, iy, iz) L / M.
#include <cmath>
#include <vector>

#include "common.cuh"

namespace dzs {

template <class R>
void fft_r2c_zy(dzs_ctx* c, const R* in, cplx<R>* out, int n, const cplx<R>* tw);

namespace {

__global__ void k_cell_start(const int32_t* __restrict__ d_n, const uint64_t* __restrict__ key, int sh,
                             int64_t ncell, int32_t* __restrict__ start) {
  const int64_t n = *d_n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t ci = (i < n) ? (int64_t)(key[i] >> sh) : ncell;
    int64_t cp = (i > 0) ? (int64_t)(key[i - 1] >> sh) : -1;
    for (int64_t q = cp + 1; q <= ci; ++q) start[q] = (int32_t)i;
  }
}

__device__ __forceinline__ uint32_t morton_cell(uint32_t x, uint32_t y, uint32_t z) {
  return (uint32_t)((spread3(x) << 2) | (spread3(y) << 1) | spread3(z));
}

template <class R>
__device__ __forceinline__ R frac32(uint32_t lo) {
  return (R)lo * (R)2.3283064365386963e-10;  // 2^-32
}

// rho[node] = sum over the 8 cells node - o, o in {0,1}^3, of k w; output
// delta.  One block per 8^3 tile of nodes: the CSR bounds of the 9^3 cells the
// tile touches are staged in shared memory once (instead of 16 scattered
// loads per node); each node then sums its 8 cells in a fixed order (cell
// offset, then particle order), so the mesh is deterministic.
template <class R>
__global__ void __launch_bounds__(256) k_cic_gather(const int32_t* __restrict__ start, const int32_t* __restrict__ d_n,
                                                    int64_t cap, const uint32_t* __restrict__ u,
                                                    const uint32_t* __restrict__ k, int M, R* __restrict__ delta,
                                                    R inv_nbar) {
  __shared__ int32_t cs[729], ce[729];
  const int T = M >> 3;
  const int tile = blockIdx.x;
  const int bx = (tile / (T * T)) * 8, by = ((tile / T) % T) * 8, bz = (tile % T) * 8;
  const int32_t n = *d_n;
  const int mask = M - 1;
  for (int q = threadIdx.x; q < 729; q += blockDim.x) {
    int i = q / 81, j = (q / 9) % 9, l = q % 9;
    uint32_t mc = morton_cell((uint32_t)((bx + i - 1) & mask), (uint32_t)((by + j - 1) & mask),
                              (uint32_t)((bz + l - 1) & mask));
    int32_t s = start[mc], e = start[mc + 1];
    s = s < 0 ? 0 : s;  // defensive: the table is consistent for sorted keys
    e = e > n ? n : e;
    cs[q] = s;
    ce[q] = e < s ? s : e;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 512; t += blockDim.x) {
    const int a = t >> 6, b = (t >> 3) & 7, c = t & 7;
    R acc = 0;
    for (int o = 0; o < 8; ++o) {
      int ox = (o >> 2) & 1, oy = (o >> 1) & 1, oz = o & 1;
      int q = (a - ox + 1) * 81 + (b - oy + 1) * 9 + (c - oz + 1);
      for (int32_t i = cs[q]; i < ce[q]; ++i) {
        R fx = frac32<R>((uint32_t)((uint64_t)u[i] * (uint64_t)M));
        R fy = frac32<R>((uint32_t)((uint64_t)u[cap + i] * (uint64_t)M));
        R fz = frac32<R>((uint32_t)((uint64_t)u[2 * cap + i] * (uint64_t)M));
        R w = (ox ? fx : (R)1 - fx) * (oy ? fy : (R)1 - fy) * (oz ? fz : (R)1 - fz);
        acc += (R)k[i] * w;
      }
    }
    delta[((int64_t)(bx + a) * M + (by + b)) * M + (bz + c)] = acc * inv_nbar - (R)1;
  }
}

// g = -grad phi (four-point stencil at the 8 surrounding nodes), CIC weights
template <class R>
__global__ void k_pm_interp(const int32_t* __restrict__ d_n, int64_t cap, const uint32_t* __restrict__ u,
                            const R* __restrict__ phi, int M, R inv12dx, R* __restrict__ g) {
  const int64_t n = *d_n;
  const int mask = M - 1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t tx = (uint64_t)u[i] * (uint64_t)M, ty = (uint64_t)u[cap + i] * (uint64_t)M,
             tz = (uint64_t)u[2 * cap + i] * (uint64_t)M;
    int bx = (int)(tx >> 32), by = (int)(ty >> 32), bz = (int)(tz >> 32);
    R fx = frac32<R>((uint32_t)tx), fy = frac32<R>((uint32_t)ty), fz = frac32<R>((uint32_t)tz);
    R ax = 0, ay = 0, az = 0;
    for (int o = 0; o < 8; ++o) {
      int ox = (o >> 2) & 1, oy = (o >> 1) & 1, oz = o & 1;
      R w = (ox ? fx : (R)1 - fx) * (oy ? fy : (R)1 - fy) * (oz ? fz : (R)1 - fz);
      int a = (bx + ox) & mask, b = (by + oy) & mask, cc = (bz + oz) & mask;
      auto P = [&](int x, int y, int z) -> R {
        return phi[((int64_t)(x & mask) * M + (y & mask)) * M + (z & mask)];
      };
      R gx = (R)8 * (P(a + 1, b, cc) - P(a - 1, b, cc)) - (P(a + 2, b, cc) - P(a - 2, b, cc));
      R gy = (R)8 * (P(a, b + 1, cc) - P(a, b - 1, cc)) - (P(a, b + 2, cc) - P(a, b - 2, cc));
      R gz = (R)8 * (P(a, b, cc + 1) - P(a, b, cc - 1)) - (P(a, b, cc + 2) - P(a, b, cc - 2));
      ax -= w * gx;
      ay -= w * gy;
      az -= w * gz;
    }
    g[i] = ax * inv12dx;
    g[cap + i] = ay * inv12dx;
    g[2 * cap + i] = az * inv12dx;
  }
}

template <class R>
void pm_impl(dzs_ctx* c, bool want_pm) {
  Buffers& B = c->B;
  const int M = c->M;
  const int64_t m3 = (int64_t)M * M * M;
  int sh = 3 * (kMaxLevel - c->logM);
  k_cell_start<<<grid_for(c->N0 + 1), kThreads, 0, c->stream>>>(B.n, B.key, sh, m3, B.cell_start);
  double n0 = (double)c->N0;
  R inv_nbar = (R)((double)m3 / n0);
  k_cic_gather<R><<<(unsigned)(m3 / 512), 256, 0, c->stream>>>(B.cell_start, B.n, c->cap, B.u, B.k, M, (R*)B.rho, inv_nbar);
  const cplx<R>* tw = (const cplx<R>*)B.twiddle;
  fft_r2c_zy<R>(c, (const R*)B.rho, (cplx<R>*)B.spec, M, tw);
  R gfac = (R)(-1.5 * c->P.omega_m / (double)m3);
  fft_c2r_3d<R>(c, (cplx<R>*)B.spec, (R*)B.phi, M, tw, (const R*)B.green_axis, gfac);
  if (want_pm) {
    R inv12dx = (R)(1.0 / (12.0 * c->P.box / M));
    k_pm_interp<R><<<grid_for(c->N0), kThreads, 0, c->stream>>>(B.n, c->cap, B.u, (const R*)B.phi, M, inv12dx,
                                                                (R*)B.g);
  }
}

}  // namespace

void launch_pm(dzs_ctx* c, bool want_pm) {
  c->launches += want_pm ? 8 : 7;
  if (c->fp64)
    pm_impl<double>(c, want_pm);
  else
    pm_impl<float>(c, want_pm);
}

template <class R>
std::vector<cplx<R>> twiddles(int n);

// twiddles of size M and the per-axis Green tables (k^2, W_CIC, r_s^2)
void launch_fft_init(dzs_ctx* c) {
  upload_fft_constants(c->dev);
  const int M = c->M;
  std::vector<double> k2(M), w(M);
  double kf = 2.0 * M_PI / c->P.box;
  for (int m = 0; m < M; ++m) {
    int s = (m <= M / 2) ? m : m - M;
    k2[m] = (kf * s) * (kf * s);
    double x = M_PI * (double)s / M;
    double sn = (s == 0) ? 1.0 : std::sin(x) / x;
    w[m] = sn * sn;
  }
  double rs2 = c->rs * c->rs;
  if (c->fp64) {
    auto tw = twiddles<double>(M);
    cudaMemcpy(c->B.twiddle, tw.data(), tw.size() * sizeof(cplx<double>), cudaMemcpyHostToDevice);
    std::vector<double> g(2 * M + 1);
    for (int m = 0; m < M; ++m) {
      g[m] = k2[m];
      g[M + m] = w[m];
    }
    g[2 * M] = rs2;
    cudaMemcpy(c->B.green_axis, g.data(), g.size() * sizeof(double), cudaMemcpyHostToDevice);
  } else {
    auto tw = twiddles<float>(M);
    cudaMemcpy(c->B.twiddle, tw.data(), tw.size() * sizeof(cplx<float>), cudaMemcpyHostToDevice);
    std::vector<float> g(2 * M + 1);
    for (int m = 0; m < M; ++m) {
      g[m] = (float)k2[m];
      g[M + m] = (float)w[m];
    }
    g[2 * M] = (float)rs2;
    cudaMemcpy(c->B.green_axis, g.data(), g.size() * sizeof(float), cudaMemcpyHostToDevice);
  }
}

}  // namespace dzs
