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
  // particle i writes i into the cells after its predecessor's cell up to its
  // own (i = n: up to the end); a lane fills a short run itself, the warp
  // fills long runs (gaps of empty cells) together, coalesced
  const int64_t n = *d_n;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; w0 <= n; w0 += stride) {
    const int64_t i = w0 + lane;
    int64_t lo = 0, hi = 0;  // cells [lo, hi) take the value i
    if (i <= n) {
      const int64_t ci = (i < n) ? (int64_t)(key[i] >> sh) : ncell;
      const int64_t cp = (i > 0) ? (int64_t)(key[i - 1] >> sh) : -1;
      lo = cp + 1;
      hi = ci + 1;
    }
    const bool longrun = hi - lo > 32;
    if (!longrun)
      for (int64_t q = lo; q < hi; ++q) start[q] = (int32_t)i;
    unsigned lm = __ballot_sync(0xffffffffu, longrun);
    while (lm) {
      const int src = __ffs(lm) - 1;
      lm &= lm - 1;
      const int64_t qlo = __shfl_sync(0xffffffffu, lo, src), qhi = __shfl_sync(0xffffffffu, hi, src);
      const int32_t v = (int32_t)__shfl_sync(0xffffffffu, i, src);
      for (int64_t q = qlo + lane; q < qhi; q += 32) start[q] = v;
    }
  }
}

__device__ __forceinline__ uint32_t morton_cell(uint32_t x, uint32_t y, uint32_t z) {
  return (uint32_t)((spread3(x) << 2) | (spread3(y) << 1) | spread3(z));
}

template <class R>
__device__ __forceinline__ R frac32(uint32_t lo) {
  return (R)lo * (R)2.3283064365386963e-10;  // 2^-32
}

// 16-byte vectors of R (aligned loads and stores of 8 weights or a phi row)
template <class R>
struct Vec16;
template <>
struct Vec16<float> {
  using T = float4;
  static constexpr int N = 4;
};
template <>
struct Vec16<double> {
  using T = double2;
  static constexpr int N = 2;
};

template <class R>
__device__ __forceinline__ void store8(R* __restrict__ dst, const R (&v)[8]) {
  using V = typename Vec16<R>::T;
  constexpr int N = Vec16<R>::N;
#pragma unroll
  for (int q = 0; q < 8 / N; ++q) {
    V x;
    R* xs = reinterpret_cast<R*>(&x);
#pragma unroll
    for (int r = 0; r < N; ++r) xs[r] = v[q * N + r];
    reinterpret_cast<V*>(dst)[q] = x;
  }
}

// W[8 i + o], i the first particle of a cell = sum over the cell's particles,
// in order, of k w_o, w_o the CIC weight of the cell's corner node
// o = (ox, oy, oz): each particle's weights are computed once (not once per
// node that reads it); the 8 sums of a cell are one aligned 8-value record
template <class R>
__global__ void k_cic_cellw(const int32_t* __restrict__ d_n, int64_t cap, const uint64_t* __restrict__ key, int sh,
                            const uint32_t* __restrict__ u, const uint32_t* __restrict__ k, int M,
                            R* __restrict__ W) {
  const int64_t n = *d_n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t c = key[i] >> sh;
    if (i > 0 && (key[i - 1] >> sh) == c) continue;  // not the first of its cell
    R acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t j = i; j < n && (key[j] >> sh) == c; ++j) {
      R fx = frac32<R>((uint32_t)((uint64_t)u[j] * (uint64_t)M));
      R fy = frac32<R>((uint32_t)((uint64_t)u[cap + j] * (uint64_t)M));
      R fz = frac32<R>((uint32_t)((uint64_t)u[2 * cap + j] * (uint64_t)M));
      const R kk = (R)k[j];
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        const int ox = (o >> 2) & 1, oy = (o >> 1) & 1, oz = o & 1;
        acc[o] += kk * ((ox ? fx : (R)1 - fx) * (oy ? fy : (R)1 - fy) * (oz ? fz : (R)1 - fz));
      }
    }
    store8(W + 8 * i, acc);
  }
}

// the same for a mesh of M = 3 2^a: particles visited in row-major cell order
// through the cell sort (sorted cell keys ck, original indices perm); W is
// indexed by the sorted position of a cell's first particle
template <class R>
__global__ void k_cic_cellw_perm(const int32_t* __restrict__ d_n, int64_t cap, const uint64_t* __restrict__ ck,
                                 const uint32_t* __restrict__ perm, const uint32_t* __restrict__ u,
                                 const uint32_t* __restrict__ k, int M, R* __restrict__ W) {
  const int64_t n = *d_n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t c = ck[t];
    if (t > 0 && ck[t - 1] == c) continue;
    R acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t s = t; s < n && ck[s] == c; ++s) {
      const int64_t j = perm[s];
      R fx = frac32<R>((uint32_t)((uint64_t)u[j] * (uint64_t)M));
      R fy = frac32<R>((uint32_t)((uint64_t)u[cap + j] * (uint64_t)M));
      R fz = frac32<R>((uint32_t)((uint64_t)u[2 * cap + j] * (uint64_t)M));
      const R kk = (R)k[j];
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        const int ox = (o >> 2) & 1, oy = (o >> 1) & 1, oz = o & 1;
        acc[o] += kk * ((ox ? fx : (R)1 - fx) * (oy ? fy : (R)1 - fy) * (oz ? fz : (R)1 - fz));
      }
    }
    store8(W + 8 * t, acc);
  }
}

__global__ void k_mesh_keys(const int32_t* __restrict__ d_n, int64_t cap, const uint32_t* __restrict__ u, int M,
                            uint64_t* __restrict__ ck) {
  const int64_t n = *d_n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t cx = ((uint64_t)u[i] * (uint64_t)M) >> 32, cy = ((uint64_t)u[cap + i] * (uint64_t)M) >> 32,
                   cz = ((uint64_t)u[2 * cap + i] * (uint64_t)M) >> 32;
    ck[i] = (cx * (uint64_t)M + cy) * (uint64_t)M + cz;
  }
}

// rho[node] = sum over the 8 cells node - o, o in {0,1}^3, of the cell's
// corner-o weight sum; output delta.  One block per 8^3 tile of nodes:
//   1. the CSR bounds of the 9^3 cells the tile touches: for Morton-ordered
//      cells the tile's own 8^3 cells are one run of the table (513
//      consecutive entries, coalesced) and only the 217 cells of the three
//      lower halo planes are looked up one by one;
//   2. each node adds the corner weight sums of its 8 cells in the fixed
//      order o = 0..7, read from the cells' records in global memory (L2;
//      empty cells add +0), so the mesh is deterministic.
template <class R, bool kMorton>
__global__ void __launch_bounds__(256) k_cic_gather(const int32_t* __restrict__ start, const int32_t* __restrict__ d_n,
                                                    const R* __restrict__ W, int M, R* __restrict__ delta,
                                                    R inv_nbar) {
  extern __shared__ unsigned char cg_raw[];
  int32_t* first = reinterpret_cast<int32_t*>(cg_raw);  // [729] first particle, -1 empty
  int32_t* sb = first + 729;                               // [513] the tile's own bounds
  const int T = M >> 3;
  const int tile = blockIdx.x;
  const int tx = tile / (T * T), ty = (tile / T) % T, tz = tile % T;
  const int bx = tx * 8, by = ty * 8, bz = tz * 8;
  const int32_t n = *d_n;
  auto clampb = [n](int32_t v) { return v < 0 ? 0 : (v > n ? n : v); };
  auto cell_of = [&](int i, int j, int l) -> int64_t {  // 9^3 coordinates (offset -1)
    if (kMorton) {  // M = 2^m: periodic wrap by a mask
      const uint32_t mk = (uint32_t)M - 1u;
      return (int64_t)morton_cell((uint32_t)(bx + i - 1) & mk, (uint32_t)(by + j - 1) & mk, (uint32_t)(bz + l - 1) & mk);
    }
    const uint32_t gx = (uint32_t)((bx + i - 1 + M) % M), gy = (uint32_t)((by + j - 1 + M) % M),
                   gz = (uint32_t)((bz + l - 1 + M) % M);
    return ((int64_t)gx * M + gy) * M + gz;
  };
  if (kMorton) {
    const int64_t base =
        (int64_t)((spread3((uint32_t)tx) << 2) | (spread3((uint32_t)ty) << 1) | spread3((uint32_t)tz)) << 9;
    for (int mo = threadIdx.x; mo <= 512; mo += blockDim.x) sb[mo] = clampb(start[base + mo]);
    for (int h = threadIdx.x; h < 217; h += blockDim.x) {
      int i, j, l;
      if (h < 81) {
        i = 0, j = h / 9, l = h % 9;
      } else if (h < 153) {
        i = 1 + (h - 81) / 9, j = 0, l = (h - 81) % 9;
      } else {
        i = 1 + (h - 153) / 8, j = 1 + (h - 153) % 8, l = 0;
      }
      const int64_t mc = cell_of(i, j, l);
      const int32_t s0 = clampb(start[mc]), e0 = clampb(start[mc + 1]);
      first[(i * 9 + j) * 9 + l] = e0 > s0 ? s0 : -1;
    }
    __syncthreads();
    for (int mo = threadIdx.x; mo < 512; mo += blockDim.x) {
      const int i = ((mo >> 6) & 4) | ((mo >> 4) & 2) | ((mo >> 2) & 1);
      const int j = ((mo >> 5) & 4) | ((mo >> 3) & 2) | ((mo >> 1) & 1);
      const int l = ((mo >> 4) & 4) | ((mo >> 2) & 2) | (mo & 1);
      first[((i + 1) * 9 + (j + 1)) * 9 + (l + 1)] = sb[mo + 1] > sb[mo] ? sb[mo] : -1;
    }
  } else {
    for (int q = threadIdx.x; q < 729; q += blockDim.x) {
      const int64_t mc = cell_of(q / 81, (q / 9) % 9, q % 9);
      const int32_t s0 = clampb(start[mc]), e0 = clampb(start[mc + 1]);
      first[q] = e0 > s0 ? s0 : -1;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 512; t += blockDim.x) {
    const int a = t >> 6, b = (t >> 3) & 7, c = t & 7;
    const int q0 = (a + 1) * 81 + (b + 1) * 9 + (c + 1);
    R acc = 0;
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      const int ox = (o >> 2) & 1, oy = (o >> 1) & 1, oz = o & 1;
      const int32_t f = first[q0 - ox * 81 - oy * 9 - oz];
      acc += f >= 0 ? W[8 * f + o] : (R)0;  // 8 f + o < 8 cap <= 2^30
    }
    delta[((int64_t)(bx + a) * M + (by + b)) * M + (bz + c)] = acc * inv_nbar - (R)1;
  }
}

template <class R>
constexpr size_t gather_smem() {
  return (729 + 513) * sizeof(int32_t);
}

// g = -grad phi at the particles for any mesh (used for M = 3 2^a): the
// four-point stencil at the 8 surrounding nodes, CIC weights, from global memory
template <class R>
__global__ void k_pm_interp(const int32_t* __restrict__ d_n, int64_t cap, const uint32_t* __restrict__ u,
                            const R* __restrict__ phi, int M, R inv12dx, R* __restrict__ g) {
  const int64_t n = *d_n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t tx = (uint64_t)u[i] * (uint64_t)M, ty = (uint64_t)u[cap + i] * (uint64_t)M,
             tz = (uint64_t)u[2 * cap + i] * (uint64_t)M;
    int bx = (int)(tx >> 32), by = (int)(ty >> 32), bz = (int)(tz >> 32);
    R fx = frac32<R>((uint32_t)tx), fy = frac32<R>((uint32_t)ty), fz = frac32<R>((uint32_t)tz);
    R ax = 0, ay = 0, az = 0;
    auto P = [&](int x, int y, int z) -> R {
      return phi[((int64_t)((x + M) % M) * M + ((y + M) % M)) * M + ((z + M) % M)];
    };
    for (int o = 0; o < 8; ++o) {
      int ox = (o >> 2) & 1, oy = (o >> 1) & 1, oz = o & 1;
      R w = (ox ? fx : (R)1 - fx) * (oy ? fy : (R)1 - fy) * (oz ? fz : (R)1 - fz);
      int a = (bx + ox) % M, b = (by + oy) % M, cc = (bz + oz) % M;
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

// g = -grad phi (four-point stencil at the 8 surrounding nodes), CIC weights.
// One block per 8^3 tile of cells = one depth-(m-3) octree cell, whose
// particles are one contiguous Morton run.  The block stages the 13^3 nodes of
// phi the tile's stencils reach as 169 rows of 16 (z from bz - 4, aligned
// 16-byte loads away from the periodic z edge), then either forms the
// gradient at the 9^3 corner nodes once (many particles) or lets each
// particle form its 8 corner gradients from the staged phi (few particles);
// both use the same four-point formula, so the result does not depend on the
// choice.
constexpr int kFlyMax = 96;  // below this many particles a tile skips the node gradients

template <class R>
__device__ __forceinline__ void grad_at(const R* __restrict__ ph, int i, int j, int l, R& gx, R& gy, R& gz) {
  // node (i, j, l) of the 9^3 corner block: phi row ((i + 2) * 13 + j + 2), z slot l + 4
  auto P = [&](int x, int y, int z) -> R { return ph[(x * 13 + y) * 16 + z]; };
  const int x = i + 2, y = j + 2, z = l + 4;
  gx = (R)8 * (P(x + 1, y, z) - P(x - 1, y, z)) - (P(x + 2, y, z) - P(x - 2, y, z));
  gy = (R)8 * (P(x, y + 1, z) - P(x, y - 1, z)) - (P(x, y + 2, z) - P(x, y - 2, z));
  gz = (R)8 * (P(x, y, z + 1) - P(x, y, z - 1)) - (P(x, y, z + 2) - P(x, y, z - 2));
}

template <class R>
__global__ void __launch_bounds__(128) k_pm_interp_tile(const int32_t* __restrict__ start, int64_t cap,
                                                        const uint32_t* __restrict__ u, const R* __restrict__ phi,
                                                        int M, R inv12dx, R* __restrict__ g) {
  extern __shared__ unsigned char pi_raw[];
  R* ph = reinterpret_cast<R*>(pi_raw);  // [169][16]: row (i, j) = node (bx - 2 + i, by - 2 + j), z = bz - 4 + slot
  R* gr = ph + 169 * 16;                 // [3][9][9][9], corner node (bx + i, ...)
  const int T = M >> 3;
  const int tile = blockIdx.x;
  const int tx = tile / (T * T), ty = (tile / T) % T, tz = tile % T;
  const int bx = tx * 8, by = ty * 8, bz = tz * 8;
  // the tile's particles: Morton prefix of the tile at depth m - 3
  const uint32_t tp = (uint32_t)((spread3((uint32_t)tx) << 2) | (spread3((uint32_t)ty) << 1) | spread3((uint32_t)tz));
  const int32_t p0 = start[(int64_t)tp << 9], p1 = start[((int64_t)tp + 1) << 9];
  if (p1 <= p0) return;  // empty tile (uniform across the block)
  const int mask = M - 1;
  if (bz >= 8 && bz + 16 <= M) {
    using V = typename Vec16<R>::T;
    constexpr int N = Vec16<R>::N, PER = 16 / N;  // vectors per row
    for (int v = threadIdx.x; v < 169 * PER; v += blockDim.x) {
      const int r = v / PER, q = v % PER;
      const int i = r / 13, j = r % 13;
      const int64_t row = ((int64_t)((bx - 2 + i) & mask) * M + ((by - 2 + j) & mask)) * M;
      reinterpret_cast<V*>(ph + r * 16)[q] = reinterpret_cast<const V*>(phi + row + bz - 4)[q];
    }
  } else {
    for (int v = threadIdx.x; v < 169 * 16; v += blockDim.x) {
      const int r = v >> 4, z = v & 15;
      const int i = r / 13, j = r % 13;
      ph[v] = phi[((int64_t)((bx - 2 + i) & mask) * M + ((by - 2 + j) & mask)) * M + ((bz - 4 + z) & mask)];
    }
  }
  __syncthreads();
  const bool fly = p1 - p0 < kFlyMax;  // uniform across the block
  if (!fly) {
    for (int q = threadIdx.x; q < 729; q += blockDim.x) {
      R gx, gy, gz;
      grad_at(ph, q / 81, (q / 9) % 9, q % 9, gx, gy, gz);
      gr[q] = gx;
      gr[729 + q] = gy;
      gr[1458 + q] = gz;
    }
    __syncthreads();
  }
  for (int64_t i = p0 + threadIdx.x; i < p1; i += blockDim.x) {
    uint64_t sx = (uint64_t)u[i] * (uint64_t)M, sy = (uint64_t)u[cap + i] * (uint64_t)M,
             sz = (uint64_t)u[2 * cap + i] * (uint64_t)M;
    // 0..7 by construction (the particle lies in the tile); clamped all the same
    const int cx = min(max((int)(sx >> 32) - bx, 0), 7), cy = min(max((int)(sy >> 32) - by, 0), 7),
              cz = min(max((int)(sz >> 32) - bz, 0), 7);
    R fx = frac32<R>((uint32_t)sx), fy = frac32<R>((uint32_t)sy), fz = frac32<R>((uint32_t)sz);
    R ax = 0, ay = 0, az = 0;
    for (int o = 0; o < 8; ++o) {
      int ox = (o >> 2) & 1, oy = (o >> 1) & 1, oz = o & 1;
      R w = (ox ? fx : (R)1 - fx) * (oy ? fy : (R)1 - fy) * (oz ? fz : (R)1 - fz);
      R gx, gy, gz;
      if (fly) {
        grad_at(ph, cx + ox, cy + oy, cz + oz, gx, gy, gz);
      } else {
        const int q = ((cx + ox) * 9 + (cy + oy)) * 9 + (cz + oz);
        gx = gr[q];
        gy = gr[729 + q];
        gz = gr[1458 + q];
      }
      ax -= w * gx;
      ay -= w * gy;
      az -= w * gz;
    }
    g[i] = ax * inv12dx;
    g[cap + i] = ay * inv12dx;
    g[2 * cap + i] = az * inv12dx;
  }
}

// the deposit reads the depth-m cell table the tree build wrote for the same keys
template <class R>
void pm_deposit(dzs_ctx* c) {
  Buffers& B = c->B;
  const int M = c->M;
  const int64_t m3 = (int64_t)M * M * M;
  double n0 = (double)c->N0;
  R inv_nbar = (R)((double)m3 / n0);
  if (c->mesh_pow2) {
    // mesh cells are the depth-m Morton cells of the tree's table
    const int sh = 3 * (kMaxLevel - c->logM);
    k_cic_cellw<R><<<grid_for(c->N0), kThreads, 0, c->stream>>>(B.n, c->cap, B.key, sh, B.u, B.k, M, (R*)B.cicw);
    k_cic_gather<R, true><<<(unsigned)(m3 / 512), 256, gather_smem<R>(), c->stream>>>(
        B.cell_start, B.n, (const R*)B.cicw, M, (R*)B.rho, inv_nbar);
    return;
  }
  // M = 3 2^a: sort the particles by row-major mesh cell (scratch: key2 and
  // prefix for the keys, idx2 and mend for the indices), CSR table of cells
  uint64_t* ka = B.key2;
  uint64_t* kb = (uint64_t*)B.prefix;
  uint32_t* va = B.idx2;
  uint32_t* vb = (uint32_t*)B.mend;
  k_mesh_keys<<<grid_for(c->N0), kThreads, 0, c->stream>>>(B.n, c->cap, B.u, M, ka);
  launch_sort_keys(c, ka, kb, va, vb, 4);  // M^3 < 2^32
  k_cell_start<<<grid_for(c->N0 + 1), kThreads, 0, c->stream>>>(B.n, ka, 0, m3, B.cell_start);
  k_cic_cellw_perm<R><<<grid_for(c->N0), kThreads, 0, c->stream>>>(B.n, c->cap, ka, va, B.u, B.k, M, (R*)B.cicw);
  k_cic_gather<R, false><<<(unsigned)(m3 / 512), 256, gather_smem<R>(), c->stream>>>(
      B.cell_start, B.n, (const R*)B.cicw, M, (R*)B.rho, inv_nbar);
}

template <class R>
void pm_fft(dzs_ctx* c) {
  Buffers& B = c->B;
  const int M = c->M;
  const int64_t m3 = (int64_t)M * M * M;
  const cplx<R>* tw = (const cplx<R>*)B.twiddle;
  fft_r2c_zy<R>(c, (const R*)B.rho, (cplx<R>*)B.spec, M, tw);
  R gfac = (R)(-1.5 * c->P.omega_m / (double)m3);
  fft_c2r_3d<R>(c, (cplx<R>*)B.spec, (R*)B.phi, M, tw, (const R*)B.green_axis, gfac);
}

template <class R>
void pm_interp(dzs_ctx* c) {
  Buffers& B = c->B;
  const int M = c->M;
  R inv12dx = (R)(1.0 / (12.0 * c->P.box / M));
  if (!c->mesh_pow2) {
    k_pm_interp<R><<<grid_for(c->N0), kThreads, 0, c->stream>>>(B.n, c->cap, B.u, (const R*)B.phi, M, inv12dx,
                                                                (R*)B.g);
    return;
  }
  const int64_t tiles = (int64_t)(M / 8) * (M / 8) * (M / 8);
  const size_t sm = (169 * 16 + 3 * 729) * sizeof(R);
  // 128 threads: a tile holds ~64 particles at the mean density, and smaller
  // blocks keep more tiles' staging loads in flight per SM
  k_pm_interp_tile<R><<<(unsigned)tiles, 128, sm, c->stream>>>(B.cell_start, c->cap, B.u, (const R*)B.phi, M,
                                                               inv12dx, (R*)B.g);
}

// ---- 3D power spectrum of the mesh (forward spectrum of the CIC delta)
//
// P_mode = |delta_k|^2 L^3 / M^6 / W(k)^2 - P_shot, W = prod_i sinc^2(pi n_i / M),
// bin b = round(|n|) decided on integers ((b - 1/2)^2 <= |n|^2 < (b + 1/2)^2),
// a half-spectrum mode with 0 < kz < M/2 standing for itself and its conjugate.
// One block per kx plane: each warp takes 32 consecutive (ky, kz) modes at a
// time; lanes of one bin are summed in lane order by their lowest lane, which
// adds to the warp's row of bins; the warps' rows are summed in warp order.
// A second pass sums the planes in kx order: deterministic.
constexpr int kPkThreads = 256;

__device__ __forceinline__ int mode_bin(int64_t n2) {
  int64_t r = (int64_t)sqrt(4.0 * (double)n2);
  while (r * r > 4 * n2) --r;
  while ((r + 1) * (r + 1) <= 4 * n2) ++r;
  return (int)((r + 1) / 2);
}

template <class R>
__global__ void k_pk_plane(const cplx<R>* __restrict__ spec, int M, const R* __restrict__ gtab, int nbins,
                           double norm, double shot, double kf, double* __restrict__ part) {
  extern __shared__ double wrow[];  // [warps][nbins][3]: modes, sum |k|, sum P
  const int kx = blockIdx.x, HN = M / 2 + 1;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int q = threadIdx.x; q < nw * nbins * 3; q += blockDim.x) wrow[q] = 0.0;
  __syncthreads();
  const int sx = kx <= M / 2 ? kx : kx - M;
  const R* wt = gtab + M;
  const int64_t nmodes = (int64_t)M * HN;
  for (int64_t base = (int64_t)w * 32; base < nmodes; base += (int64_t)nw * 32) {
    const int64_t q = base + lane;
    int b = 0;
    double cnt = 0.0, ksum = 0.0, psum = 0.0;
    if (q < nmodes) {
      const int ky = (int)(q / HN), kz = (int)(q % HN);
      const int sy = ky <= M / 2 ? ky : ky - M;
      const int64_t n2 = (int64_t)sx * sx + (int64_t)sy * sy + (int64_t)kz * kz;
      b = mode_bin(n2);
      if (b >= 1 && b <= nbins) {
        const cplx<R> d = spec[((int64_t)kx * M + ky) * HN + kz];
        const double wv = (double)wt[kx] * (double)wt[ky] * (double)wt[kz];
        const double p = ((double)d.x * (double)d.x + (double)d.y * (double)d.y) * norm / (wv * wv) - shot;
        cnt = (kz == 0 || 2 * kz == M) ? 1.0 : 2.0;
        ksum = cnt * kf * sqrt((double)n2);
        psum = cnt * p;
      } else {
        b = 0;
      }
    }
    const unsigned same = __match_any_sync(0xffffffffu, b);
    const int lead = __ffs(same) - 1;
    double c = 0.0, ks = 0.0, ps = 0.0;
    for (int l = 0; l < 32; ++l) {  // every lane joins each shuffle; the leader keeps its bin's lanes
      const double tc = __shfl_sync(0xffffffffu, cnt, l), tk = __shfl_sync(0xffffffffu, ksum, l),
                   tp = __shfl_sync(0xffffffffu, psum, l);
      if ((same >> l) & 1u) {
        c += tc;
        ks += tk;
        ps += tp;
      }
    }
    if (lane == lead && b >= 1) {
      double* row = wrow + ((int64_t)w * nbins + (b - 1)) * 3;
      row[0] += c;
      row[1] += ks;
      row[2] += ps;
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nbins * 3; q += blockDim.x) {
    double s = 0.0;
    for (int v = 0; v < nw; ++v) s += wrow[(int64_t)v * nbins * 3 + q];
    part[(int64_t)kx * nbins * 3 + q] = s;
  }
}

__global__ void k_pk_final(const double* __restrict__ part, int M, int nbins, double* __restrict__ out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;  // (bin, field)
  if (q >= nbins * 3) return;
  double s = 0.0;
  for (int kx = 0; kx < M; ++kx) s += part[(int64_t)kx * nbins * 3 + q];
  out[q] = s;
}

__global__ void k_sum_k2(const int32_t* __restrict__ d_n, const uint32_t* __restrict__ k,
                         unsigned long long* __restrict__ out) {
  const int64_t n = *d_n;
  unsigned long long s = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += (unsigned long long)k[i] * k[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

template <class R>
void pm_deposit(dzs_ctx* c);

template <class R>
void pk_impl(dzs_ctx* c, int nbins, double* d_part, double* d_out, double shot) {
  Buffers& B = c->B;
  const int M = c->M;
  const int64_t m3 = (int64_t)M * M * M;
  launch_cell_start(c);
  pm_deposit<R>(c);
  fft_r2c_3d<R>(c, (const R*)B.rho, (cplx<R>*)B.spec, M, (const cplx<R>*)B.twiddle);
  const double L = c->P.box;
  const double norm = L * L * L / ((double)m3 * (double)m3);
  const size_t smem = (size_t)(kPkThreads / 32) * nbins * 3 * sizeof(double);
  k_pk_plane<R><<<M, kPkThreads, smem, c->stream>>>((const cplx<R>*)B.spec, M, (const R*)B.green_axis, nbins, norm,
                                                    shot, 2.0 * M_PI / L, d_part);
  k_pk_final<<<(nbins * 3 + 255) / 256, 256, 0, c->stream>>>(d_part, M, nbins, d_out);
}

}  // namespace

// P(k) of the current particles: sums of [modes, |k|, P] per bin in d_out
// [nbins][3]; d_part holds M * nbins * 3 doubles.  The state must be
// Morton-sorted with valid keys.
void launch_pk(dzs_ctx* c, int nbins, double* d_part, double* d_out, double shot) {
  c->launches += c->mesh_pow2 ? 8 : 21;
  if (c->fp64)
    pk_impl<double>(c, nbins, d_part, d_out, shot);
  else
    pk_impl<float>(c, nbins, d_part, d_out, shot);
}

void launch_sum_k2(dzs_ctx* c, unsigned long long* out) {
  c->launches += 1;
  cudaMemsetAsync(out, 0, sizeof(unsigned long long), c->stream);
  k_sum_k2<<<grid_for(c->N0), kThreads, 0, c->stream>>>(c->B.n, c->B.k, out);
}

// the PM force in three stages: CIC deposit of delta; FFT Poisson solve with
// the Green function fused into the X pass (phi); four-point gradient and
// CIC interpolation to the particles (g)
// CSR table of the depth-m Morton cells (m = log2 M) of the current keys
void launch_cell_start(dzs_ctx* c) {
  c->launches += 1;
  const int64_t ncell = (int64_t)1 << (3 * c->logM);  // M^3 for M = 2^m
  const int sh = 3 * (kMaxLevel - c->logM);
  k_cell_start<<<grid_for(c->N0 + 1), kThreads, 0, c->stream>>>(c->B.n, c->B.key, sh, ncell, c->B.cell_start);
}

void launch_pm_deposit(dzs_ctx* c) {
  c->launches += c->mesh_pow2 ? 2 : 16;
  if (c->fp64)
    pm_deposit<double>(c);
  else
    pm_deposit<float>(c);
}

void launch_pm_fft(dzs_ctx* c) {
  c->launches += 5;
  if (c->fp64)
    pm_fft<double>(c);
  else
    pm_fft<float>(c);
}

void launch_pm_interp(dzs_ctx* c) {
  c->launches += 1;
  if (c->fp64)
    pm_interp<double>(c);
  else
    pm_interp<float>(c);
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
