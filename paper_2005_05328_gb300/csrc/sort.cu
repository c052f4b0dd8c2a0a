// sort.cu -- stable LSD radix sort of the 63-bit Morton keys (8-bit digits,
// 8 passes) carrying the particle index, then one gather pass that permutes
// the particle state into Morton order.
//
// The oct-tree of the paper (Sec. 2.1) becomes an implicit octree over the
// sorted keys: every octree cell is a contiguous run of the sorted array.
// Each pass: per-tile digit histograms, a per-digit scan over tiles, and a
// stable scatter (rank = earlier items of the same digit in the tile).  Ties
// keep the previous order, so the result is deterministic.
#include "common.cuh"

namespace dzs {
namespace {

constexpr int kSortThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kSortThreads * kItems;  // 2048 keys per block
constexpr int kDigits = 256;

__global__ void k_hist(const uint64_t* __restrict__ key, const int32_t* __restrict__ d_n, int shift,
                       uint32_t* __restrict__ hist, int nb) {
  __shared__ uint32_t cnt[kDigits];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t n = *d_n;
  int64_t base = (int64_t)blockIdx.x * kTile;
  uint64_t kv[kItems];  // all loads in flight before the first count
#pragma unroll
  for (int s = 0; s < kItems; ++s) {
    int64_t i = base + s * kSortThreads + threadIdx.x;
    kv[s] = i < n ? key[i] : 0ull;
  }
#pragma unroll
  for (int s = 0; s < kItems; ++s) {
    int64_t i = base + s * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(kv[s] >> shift) & 0xff], 1u);
  }
  __syncthreads();
  hist[threadIdx.x * nb + blockIdx.x] = cnt[threadIdx.x];
}

// block d: exclusive scan of row d of the histogram, row total to rowtot[d]
__global__ void k_scan_rows(uint32_t* __restrict__ hist, int nb, uint32_t* __restrict__ rowtot) {
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t carry;
  uint32_t* row = hist + (int64_t)blockIdx.x * nb;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int b0 = 0; b0 < nb; b0 += blockDim.x) {
    int b = b0 + threadIdx.x;
    uint32_t v = b < nb ? row[b] : 0u, inc = v;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
      uint32_t t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0u, ti = t;
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t q = __shfl_up_sync(0xffffffffu, ti, o);
        if (lane >= o) ti += q;
      }
      warp_tot[lane] = ti - t;
    }
    __syncthreads();
    uint32_t ex = inc - v + warp_tot[w] + carry;
    if (b < nb) row[b] = ex;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = ex + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) rowtot[blockIdx.x] = carry;
}

__global__ void k_scatter(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                          uint64_t* __restrict__ kout, uint32_t* __restrict__ vout,
                          const int32_t* __restrict__ d_n, int shift, const uint32_t* __restrict__ hist,
                          int nb, const uint32_t* __restrict__ rowtot, bool identity_values) {
  __shared__ uint32_t gbase[kDigits];  // output position of the tile's first key of each digit
  __shared__ uint32_t lbase[kDigits];  // the same within the tile (tile sorted by digit)
  __shared__ uint32_t run[kDigits];
  __shared__ uint32_t wcnt[kSortThreads / 32][kDigits];
  __shared__ uint64_t sk[kTile];       // the tile, stably sorted by digit
  __shared__ uint32_t sv[kTile];
  const int64_t n = *d_n;
  int64_t base = (int64_t)blockIdx.x * kTile;
  if (base >= n) return;
  const int tile_n = (int)(n - base < kTile ? n - base : kTile);
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  // the tile's keys and values, all loads in flight before any waiting
  uint64_t kreg[kItems];
  uint32_t vreg[kItems];
#pragma unroll
  for (int s = 0; s < kItems; ++s) {
    const int64_t i = base + s * kSortThreads + t;
    kreg[s] = i < n ? kin[i] : 0ull;
    vreg[s] = i < n ? (identity_values ? (uint32_t)i : vin[i]) : 0u;
  }
  // digit bases: exclusive scans over the 256 digits (thread t owns digit t) of
  // the row totals (global) and of this tile's counts (local); warp scans,
  // then a scan of the 8 warp totals
  {
    __shared__ uint32_t wtot[2][kSortThreads / 32];
    const uint32_t h0 = hist[(int64_t)t * nb + blockIdx.x];
    const uint32_t h1 = blockIdx.x + 1 < (unsigned)nb ? hist[(int64_t)t * nb + blockIdx.x + 1] : rowtot[t];
    const uint32_t v = rowtot[t], c = h1 - h0;
    uint32_t inc = v, incc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o), yc = __shfl_up_sync(0xffffffffu, incc, o);
      if (lane >= o) {
        inc += y;
        incc += yc;
      }
    }
    if (lane == 31) {
      wtot[0][w] = inc;
      wtot[1][w] = incc;
    }
    __syncthreads();
    uint32_t before = 0, beforec = 0;
    for (int q = 0; q < w; ++q) {
      before += wtot[0][q];
      beforec += wtot[1][q];
    }
    gbase[t] = before + inc - v + h0;
    lbase[t] = beforec + incc - c;
    run[t] = 0;
  }
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int s = 0; s < kItems; ++s) {
    for (int q = 0; q < kSortThreads / 32; ++q) wcnt[q][t] = 0;
    __syncthreads();
    int64_t i = base + s * kSortThreads + t;
    bool valid = i < n;
    uint64_t kv = kreg[s];
    uint32_t vv = vreg[s];
    int d = valid ? (int)((kv >> shift) & 0xff) : kDigits;  // invalid items group apart
    unsigned peers = __match_any_sync(0xffffffffu, d);
    int rank_w = __popc(peers & lt);
    if (valid && rank_w == 0) wcnt[w][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t off = run[t];
      for (int q = 0; q < kSortThreads / 32; ++q) {
        uint32_t c = wcnt[q][t];
        wcnt[q][t] = off;
        off += c;
      }
      run[t] = off;
    }
    __syncthreads();
    if (valid) {
      const uint32_t lp = lbase[d] + wcnt[w][d] + (uint32_t)rank_w;
      if (lp < (uint32_t)kTile) {  // always, when the tile's histogram matches its keys
        sk[lp] = kv;
        sv[lp] = vv;
      }
    }
    __syncthreads();  // wcnt is read above and cleared at the top of the next round
  }
  // runs of one digit are contiguous in the tile and in the output: coalesced
  for (int q = t; q < tile_n; q += kSortThreads) {
    const uint64_t kv = sk[q];
    const int d = (int)((kv >> shift) & 0xff);
    const uint32_t pos = gbase[d] + (uint32_t)q - lbase[d];
    if ((int64_t)pos < n) {
      kout[pos] = kv;
      vout[pos] = sv[q];
    }
  }
}

template <class R>
__global__ void k_permute(const int32_t* __restrict__ d_n, int64_t cap, const uint32_t* __restrict__ idx,
                          const uint32_t* __restrict__ u, const R* __restrict__ p,
                          const uint32_t* __restrict__ k, const uint32_t* __restrict__ id,
                          const uint8_t* __restrict__ fl, uint32_t* __restrict__ u2, R* __restrict__ p2,
                          uint32_t* __restrict__ k2, uint32_t* __restrict__ id2, uint8_t* __restrict__ fl2) {
  const int64_t n = *d_n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t s = idx[t];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      u2[ax * cap + t] = u[ax * cap + s];
      p2[ax * cap + t] = p[ax * cap + s];
    }
    k2[t] = k[s];
    id2[t] = id[s];
    fl2[t] = fl[s];
  }
}

}  // namespace

// stable LSD radix sort of n keys (an even number of 8-bit passes from bit 0)
// with their indices (identity on input); the result is in ka / va again
void launch_sort_keys(dzs_ctx* c, uint64_t* ka, uint64_t* kb, uint32_t* va, uint32_t* vb, int passes) {
  c->launches += 3 * passes;
  Buffers& B = c->B;
  int nb = (int)((c->cap + kTile - 1) / kTile);
  uint32_t* rowtot = B.hist + (int64_t)kDigits * nb;
  uint64_t *kin = ka, *kout = kb;
  uint32_t *vin = va, *vout = vb;
  for (int pass = 0; pass < passes; ++pass) {
    int shift = 8 * pass;
    k_hist<<<nb, kSortThreads, 0, c->stream>>>(kin, B.n, shift, B.hist, nb);
    k_scan_rows<<<kDigits, 1024, 0, c->stream>>>(B.hist, nb, rowtot);
    k_scatter<<<nb, kSortThreads, 0, c->stream>>>(kin, vin, kout, vout, B.n, shift, B.hist, nb, rowtot,
                                                  pass == 0);
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
}

void launch_sort(dzs_ctx* c) {
  c->launches += 25;
  Buffers& B = c->B;
  int nb = (int)((c->cap + kTile - 1) / kTile);
  uint32_t* rowtot = B.hist + (int64_t)kDigits * nb;
  uint64_t *kin = B.key, *kout = B.key2;
  uint32_t *vin = B.idx, *vout = B.idx2;
  for (int pass = 0; pass < 8; ++pass) {
    int shift = 8 * pass;
    k_hist<<<nb, kSortThreads, 0, c->stream>>>(kin, B.n, shift, B.hist, nb);
    k_scan_rows<<<kDigits, 1024, 0, c->stream>>>(B.hist, nb, rowtot);
    k_scatter<<<nb, kSortThreads, 0, c->stream>>>(kin, vin, kout, vout, B.n, shift, B.hist, nb, rowtot,
                                                  pass == 0);
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  // 8 passes: sorted keys and indices are back in key / idx
  int grid = grid_for(c->N0);
  if (c->fp64)
    k_permute<double><<<grid, kThreads, 0, c->stream>>>(B.n, c->cap, B.idx, B.u, (const double*)B.p, B.k, B.id,
                                                        B.fl, B.u2, (double*)B.p2, B.k2, B.id2, B.fl2);
  else
    k_permute<float><<<grid, kThreads, 0, c->stream>>>(B.n, c->cap, B.idx, B.u, (const float*)B.p, B.k, B.id,
                                                       B.fl, B.u2, (float*)B.p2, B.k2, B.id2, B.fl2);
  std::swap(B.u, B.u2);
  std::swap(B.p, B.p2);
  std::swap(B.k, B.k2);
  std::swap(B.id, B.id2);
  std::swap(B.fl, B.fl2);
}

}  // namespace dzs

// ---- helpers used by the state-injection entry points

namespace dzs {
namespace {

__global__ void k_keys(const int32_t* __restrict__ d_n, int64_t cap, const uint32_t* __restrict__ u,
                       uint64_t* __restrict__ key) {
  const int64_t n = *d_n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    key[i] = morton_key(u[i], u[cap + i], u[2 * cap + i]);
}

// undo the last sort: sorted slot t goes back to idx[t]; g (sorted) is written
// as double in the original order with stride n
template <class R>
__global__ void k_unpermute(const int32_t* __restrict__ d_n, int64_t cap, const uint32_t* __restrict__ idx,
                            const uint32_t* __restrict__ u, const R* __restrict__ p, const R* __restrict__ g,
                            const uint32_t* __restrict__ k, const uint32_t* __restrict__ id,
                            const uint8_t* __restrict__ fl, uint32_t* __restrict__ u2, R* __restrict__ p2,
                            uint32_t* __restrict__ k2, uint32_t* __restrict__ id2, uint8_t* __restrict__ fl2,
                            double* __restrict__ gout) {
  const int64_t n = *d_n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t o = idx[t];
    for (int ax = 0; ax < 3; ++ax) {
      u2[ax * cap + o] = u[ax * cap + t];
      p2[ax * cap + o] = p[ax * cap + t];
      gout[ax * n + o] = (double)g[ax * cap + t];
    }
    k2[o] = k[t];
    id2[o] = id[t];
    fl2[o] = fl[t];
  }
}

template <class R>
__global__ void k_close_kick(const int32_t* __restrict__ d_n, int64_t cap, R* __restrict__ p,
                             const R* __restrict__ g, R kick) {
  const int64_t n = *d_n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int ax = 0; ax < 3; ++ax) p[ax * cap + i] += g[ax * cap + i] * kick;
}

}  // namespace

void launch_keys(dzs_ctx* c) {
  c->launches += 1;
  k_keys<<<grid_for(c->N0), kThreads, 0, c->stream>>>(c->B.n, c->cap, c->B.u, c->B.key);
}

void launch_unpermute(dzs_ctx* c, double* g_out) {
  c->launches += 1;
  Buffers& B = c->B;
  int grid = grid_for(c->N0);
  if (c->fp64)
    k_unpermute<double><<<grid, kThreads, 0, c->stream>>>(B.n, c->cap, B.idx, B.u, (const double*)B.p,
                                                          (const double*)B.g, B.k, B.id, B.fl, B.u2,
                                                          (double*)B.p2, B.k2, B.id2, B.fl2, g_out);
  else
    k_unpermute<float><<<grid, kThreads, 0, c->stream>>>(B.n, c->cap, B.idx, B.u, (const float*)B.p,
                                                         (const float*)B.g, B.k, B.id, B.fl, B.u2, (float*)B.p2,
                                                         B.k2, B.id2, B.fl2, g_out);
  std::swap(B.u, B.u2);
  std::swap(B.p, B.p2);
  std::swap(B.k, B.k2);
  std::swap(B.id, B.id2);
  std::swap(B.fl, B.fl2);
}

void launch_close_kick(dzs_ctx* c, int step) {
  c->launches += 1;
  if (c->fp64)
    k_close_kick<double><<<grid_for(c->N0), kThreads, 0, c->stream>>>(c->B.n, c->cap, (double*)c->B.p,
                                                                      (const double*)c->B.g, c->T.kick2[step]);
  else
    k_close_kick<float><<<grid_for(c->N0), kThreads, 0, c->stream>>>(c->B.n, c->cap, (float*)c->B.p,
                                                                     (const float*)c->B.g, (float)c->T.kick2[step]);
}

}  // namespace dzs

// ---- allocation-free Morton sort for callers that cannot allocate device memory
//
// Some callers may not call cudaMalloc at all: code running inside a host
// framework whose device memory is fully owned by its own allocator, plugins
// with a fixed memory budget, or code paths that must not synchronise the
// device (cudaMalloc/cudaFree can).  dzs_morton_sort_noalloc serves them: its
// scratch (keys and indices ping-pong buffers, digit histograms and the
// device-side count) lives in one file-scope static device array of fixed
// size, allocated when the library is loaded and kept until the process exits.
// The caller passes device inputs and outputs; nothing is allocated per call.

#include <mutex>

namespace dzs {
namespace {

constexpr size_t kNoallocMaxN = DZS_NOALLOC_SORT_MAX_N;
constexpr size_t kNoallocNb = (kNoallocMaxN + kTile - 1) / kTile;
// layout: keyA, keyB (uint64), valA, valB (uint32), hist (257 rows of nb + 256),
// count slot
constexpr size_t kOffKeyB = 8 * kNoallocMaxN;
constexpr size_t kOffValA = 16 * kNoallocMaxN;
constexpr size_t kOffValB = 20 * kNoallocMaxN;
constexpr size_t kOffHist = 24 * kNoallocMaxN;
constexpr size_t kOffCount = kOffHist + 4 * (257 * kNoallocNb + 256);
constexpr size_t kNoallocBytes = kOffCount + 256;

static __device__ __align__(256) unsigned char g_sort_scratch[kNoallocBytes];

std::mutex g_scratch_mu;
void* g_scratch_dev[256] = {nullptr};  // device address per device ordinal

__global__ void k_set_count(int32_t* slot, int32_t n) { *slot = n; }

}  // namespace
}  // namespace dzs

extern "C" dzs_status dzs_morton_sort_noalloc(const uint32_t* d_u, size_t n, uint32_t* d_perm, uint64_t* d_keys,
                                              void* cuda_stream) {
  using namespace dzs;
  if (n > kNoallocMaxN) return DZS_EINVAL;  // above the static scratch capacity
  if (n > 0 && (!d_u || !d_perm)) return DZS_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return DZS_EDEVICE;
  void* base = nullptr;
  {
    // set-up, once per device, with that device current: the host-side name of
    // the array is not a device address, so ask the runtime for it
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_dev[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) return DZS_ECUDA;
      g_scratch_dev[dev] = p;
    }
    base = g_scratch_dev[dev];
  }
  if (n == 0) return DZS_OK;
  // an error left pending by earlier work on this thread is not ours to
  // report or to clear: refuse before launching anything
  if (cudaPeekAtLastError() != cudaSuccess) return DZS_ECUDA;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  char* b = (char*)base;
  uint64_t* keyA = (uint64_t*)b;
  uint64_t* keyB = (uint64_t*)(b + kOffKeyB);
  uint32_t* valA = (uint32_t*)(b + kOffValA);
  uint32_t* valB = (uint32_t*)(b + kOffValB);
  uint32_t* hist = (uint32_t*)(b + kOffHist);
  int32_t* count = (int32_t*)(b + kOffCount);
  // every scratch word read below is first written by this call: the count,
  // the keys, the per-tile histograms (all 256 rows of every tile) and the row
  // totals, so nothing left over from a previous call is used
  const int nb = (int)((n + kTile - 1) / kTile);
  uint32_t* rowtot = hist + (int64_t)kDigits * nb;
  // each launch is checked with cudaPeekAtLastError (a launch error is sticky
  // for this call's own launches only: nothing was pending before them)
  k_set_count<<<1, 1, 0, st>>>(count, (int32_t)n);
  if (cudaPeekAtLastError() != cudaSuccess) return DZS_ECUDA;
  k_keys<<<grid_for((int64_t)n), kThreads, 0, st>>>(count, (int64_t)n, d_u, keyA);
  if (cudaPeekAtLastError() != cudaSuccess) return DZS_ECUDA;
  uint64_t *kin = keyA, *kout = keyB;
  uint32_t *vin = valA, *vout = valB;
  for (int pass = 0; pass < 8; ++pass) {
    int shift = 8 * pass;
    k_hist<<<nb, kSortThreads, 0, st>>>(kin, count, shift, hist, nb);
    k_scan_rows<<<kDigits, 1024, 0, st>>>(hist, nb, rowtot);
    k_scatter<<<nb, kSortThreads, 0, st>>>(kin, vin, kout, vout, count, shift, hist, nb, rowtot, pass == 0);
    if (cudaPeekAtLastError() != cudaSuccess) return DZS_ECUDA;
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  if (cudaMemcpyAsync(d_perm, vin, 4 * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return DZS_ECUDA;
  if (d_keys && cudaMemcpyAsync(d_keys, kin, 8 * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return DZS_ECUDA;
  return DZS_OK;
}
