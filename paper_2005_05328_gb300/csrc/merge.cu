// merge.cu -- the DZS de-refinement (paper Sec. 2.2, Fig. 2; Eq. 3;
// Sec. 2.2.1 geometric criterion with the l_max limit).
//
// GPU formulation of the top-down walk: every octree cell is a run of the
// Morton-sorted particles, and its mass and mass-weighted position are exact
// differences of uint64 prefix sums (masses are integer multiples of m0, so
// the sums are exact in any order).  Each particle walks its own root-to-leaf
// path from the coarsest candidate level j_min (side <= l_max), locating its
// cell by binary search inside the parent's range, and stops at the first
// cell with >= 2 particles that qualifies:
//     d_COM^2 > T_j^2,   T_j = R_lat + b_lat + ceil(l_j / theta_dzs),
// which is l_j / D_n < theta_dzs with D_n = d_COM - R_lc - b (Eq. 3).  Every
// member reaches the same decision, so the walk needs no synchronisation.
// The first member of a merged cell becomes the new particle (mass K, integer
// COM rounded half up, p = (sum k p) / K summed left to right in FP64,
// id = min id); the others are dropped by a stable compaction.
//
// Dynamical criterion (Sec. 2.2.1: Eq. 2 with d replaced by D_n of Eq. 3 and
// |a_old| by the smallest |a| of the particles not yet crossed): merge iff
//     D > 0  and  G M l_j^2 / D^4 < alpha a_min,
//     D = (sqrt(d_COM^2) - (R_lat + b_lat)) L / 2^32,
// every operation a correctly rounded FP64 intrinsic in that order, so the
// decision equals a plain IEEE evaluation bit for bit.  a_min^2 is reduced
// on the device just before the mark pass from the accelerations the state
// carries (the previous step's forces) and the crossing flags of this step.
//
// Steps where little can merge cost little: a level whose T_j is beyond the
// largest possible COM distance (the box corner) is never tested, and with
// the geometric criterion (members must lie beyond R_lat + b_lat) a first
// mark pass sums the few particles of each candidate cell directly; only when
// some candidate cell holds more than kDirect particles are the prefix sums
// built and those candidates marked again from them (same decisions: the sums
// are exact either way).  The compaction writes only from the first particle
// that changes, into the spare arrays, and copies that tail back: a step that
// merges nothing writes nothing.
#include <cmath>

#include "common.cuh"

namespace dzs {
namespace {

constexpr int kChunk = 1024;
constexpr int kDirect = 64;              // largest cell the first mark pass sums directly
constexpr int32_t kDeferred = INT32_MIN;  // mend of a candidate left to the prefix pass

struct MergeParams {
  uint64_t thr[kMaxLevel + 1];  // T_j (UINT64_MAX: level never merges)
  uint64_t rb2;                 // (R_lat + b_lat)^2: members must lie beyond
  int jmin;
  int jstart;                   // first level that can merge (>= max(jmin, 1))
  int filter;                   // 1 when theta_dzs <= 1/sqrt(3) (geometric only)
  int criterion;                // DZS_CRIT_GEOMETRIC / DZS_CRIT_DYNAMICAL
  double rb;                    // R_lat + b_lat (dynamical)
  double scale;                 // L / 2^32
  double gm0;                   // G m0 = 1.5 Omega_m L^3 / (4 pi N0)
  double alpha;                 // alpha of Eq. 2
  double l2[kMaxLevel + 1];     // (L / 2^j)^2
  const uint64_t* amin2_slot;   // ~bits of a_min^2 (0: no particle inside)
};

// a_min^2 = min over particles not yet crossed of |g|^2, FP64 without
// contraction.  Non-negative doubles order like their bit patterns, so the
// minimum is an integer max over the complemented bits (slot zeroed before).
template <class R>
__global__ void k_amin2(const int32_t* __restrict__ d_n, int64_t cap, const R* __restrict__ g,
                        const uint8_t* __restrict__ fl, unsigned long long* __restrict__ slot) {
  const int64_t n = *d_n;
  unsigned long long best = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (fl[i] & kFlCrossed) continue;
    double gx = (double)g[i], gy = (double)g[cap + i], gz = (double)g[2 * cap + i];
    double a2 = __dadd_rn(__dadd_rn(__dmul_rn(gx, gx), __dmul_rn(gy, gy)), __dmul_rn(gz, gz));
    if (!(a2 == a2)) continue;  // NaN never wins the minimum
    unsigned long long c = ~(unsigned long long)__double_as_longlong(a2);
    best = c > best ? c : best;
  }
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long t = __shfl_down_sync(0xffffffffu, best, o);
    best = t > best ? t : best;
  }
  __shared__ unsigned long long wbest[32];
  if ((threadIdx.x & 31) == 0) wbest[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x < 32) {
    best = threadIdx.x < (blockDim.x >> 5) ? wbest[threadIdx.x] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long t = __shfl_down_sync(0xffffffffu, best, o);
      best = t > best ? t : best;
    }
    if (threadIdx.x == 0 && best) atomicMax(slot, best);  // one atomic per block
  }
}

__device__ __forceinline__ bool dynamical_merge(const MergeParams& mp, uint64_t d2, uint64_t K, int j,
                                                double rhs) {
  double D = __dmul_rn(__dsub_rn(__dsqrt_rn((double)d2), mp.rb), mp.scale);
  if (!(D > 0.0)) return false;
  double D2 = __dmul_rn(D, D);
  double lhs = __ddiv_rn(__dmul_rn(__dmul_rn(mp.gm0, (double)K), mp.l2[j]), __dmul_rn(D2, D2));
  return lhs < rhs;
}

// ---- 4-channel uint64 exclusive prefix sums: k, k ux, k uy, k uz
__global__ void k_prefix_totals(const int32_t* __restrict__ d_n, int64_t cap, const uint32_t* __restrict__ u,
                                const uint32_t* __restrict__ k, uint64_t* __restrict__ tot,
                                const unsigned* __restrict__ need) {
  if (need && !*need) return;
  const int64_t n = *d_n;
  int64_t base = (int64_t)blockIdx.x * kChunk;
  unsigned long long s[4] = {0, 0, 0, 0};
  for (int t = threadIdx.x; t < kChunk; t += blockDim.x) {
    int64_t i = base + t;
    if (i < n) {
      uint64_t kk = k[i];
      s[0] += kk;
      for (int ax = 0; ax < 3; ++ax) s[1 + ax] += kk * u[ax * cap + i];
    }
  }
  for (int q = 0; q < 4; ++q) {
    for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_down_sync(0xffffffffu, s[q], o);
  }
  __shared__ unsigned long long ws[4][32];
  if ((threadIdx.x & 31) == 0)
    for (int q = 0; q < 4; ++q) ws[q][threadIdx.x >> 5] = s[q];
  __syncthreads();
  if (threadIdx.x < 4) {
    unsigned long long a = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += ws[threadIdx.x][w];
    tot[(int64_t)threadIdx.x * (gridDim.x + 1) + blockIdx.x] = a;
  }
}

// block c scans row c (channel c) of the chunk totals, 1024 at a time
__global__ void k_prefix_scan_totals(uint64_t* __restrict__ tot, int nchunks, const unsigned* __restrict__ need) {
  if (need && !*need) return;
  __shared__ unsigned long long woff[32];
  __shared__ unsigned long long carry, block_total;
  uint64_t* row = tot + (int64_t)blockIdx.x * (nchunks + 1);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nchunks; base += blockDim.x) {
    int i = base + threadIdx.x;
    unsigned long long v = i < nchunks ? row[i] : 0ull, inc = v;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) woff[w] = inc;
    __syncthreads();
    if (w == 0) {
      unsigned long long t = lane < nw ? woff[lane] : 0ull, ti = t;
      for (int o = 1; o < 32; o <<= 1) {
        unsigned long long q = __shfl_up_sync(0xffffffffu, ti, o);
        if (lane >= o) ti += q;
      }
      if (lane < nw) woff[lane] = ti - t;
      if (lane == nw - 1) block_total = ti;
    }
    __syncthreads();
    if (i < nchunks) row[i] = carry + woff[w] + inc - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += block_total;
    __syncthreads();
  }
  if (threadIdx.x == 0) row[nchunks] = carry;
}

__global__ void k_prefix_apply(const int32_t* __restrict__ d_n, int64_t cap, const uint32_t* __restrict__ u,
                               const uint32_t* __restrict__ k, const uint64_t* __restrict__ tot, int nchunks,
                               uint64_t* __restrict__ pre, const unsigned* __restrict__ need) {
  if (need && !*need) return;
  const int64_t n = *d_n;
  int64_t base = (int64_t)blockIdx.x * kChunk;
  if (base > n) return;
  // thread t owns items base + 4t .. base + 4t + 3
  int64_t i0 = base + 4 * threadIdx.x;
  unsigned long long v[4][4], s[4] = {0, 0, 0, 0};
  for (int q = 0; q < 4; ++q) {
    int64_t i = i0 + q;
    uint64_t kk = (i < n) ? k[i] : 0;
    v[0][q] = kk;
    for (int ax = 0; ax < 3; ++ax) v[1 + ax][q] = (i < n) ? kk * u[ax * cap + i] : 0;
    for (int c = 0; c < 4; ++c) s[c] += v[c][q];
  }
  // block exclusive scan per channel (warp shuffles + warp totals)
  __shared__ unsigned long long wt[4][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned long long inc[4];
  for (int c = 0; c < 4; ++c) {
    inc[c] = s[c];
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long t = __shfl_up_sync(0xffffffffu, inc[c], o);
      if (lane >= o) inc[c] += t;
    }
    if (lane == 31) wt[c][w] = inc[c];
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    unsigned long long a = 0;
    for (int q = 0; q < nw; ++q) {
      unsigned long long t = wt[threadIdx.x][q];
      wt[threadIdx.x][q] = a;
      a += t;
    }
  }
  __syncthreads();
  for (int c = 0; c < 4; ++c) {
    unsigned long long run = tot[(int64_t)c * (nchunks + 1) + blockIdx.x] + wt[c][w] + inc[c] - s[c];
    for (int q = 0; q < 4; ++q) {
      int64_t i = i0 + q;
      if (i <= n) pre[(int64_t)c * (cap + 1) + i] = run;
      run += v[c][q];
    }
  }
}

__device__ __forceinline__ int64_t lower_bound_key(const uint64_t* __restrict__ key, int64_t lo, int64_t hi,
                                                   uint64_t x) {
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (key[mid] < x)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// mend[i]: end of the merged run if i leads one, -1 if i is merged away, 0 if kept
// first index s <= i with key[s] >= x, given key[i] >= x: exponential steps
// down from i, then a binary search of the last step (cost ~2 log2(i - s))
__device__ __forceinline__ int64_t gallop_down(const uint64_t* __restrict__ key, int64_t i, uint64_t x) {
  int64_t hi = i, lo = 0;
  for (int64_t step = 1;; step <<= 1) {
    const int64_t p = i - step;
    if (p < 0) break;
    if (key[p] < x) {
      lo = p + 1;
      break;
    }
    hi = p;
  }
  return lower_bound_key(key, lo, hi + 1, x);
}

// first index >= i1 with key >= x (or n), given key[i1 - 1] < x
__device__ __forceinline__ int64_t gallop_up(const uint64_t* __restrict__ key, int64_t i1, int64_t n, uint64_t x) {
  int64_t lo = i1, hi = n;
  for (int64_t step = 1;; step <<= 1) {
    const int64_t p = i1 - 1 + step;
    if (p >= n) break;
    if (key[p] >= x) {
      hi = p;
      break;
    }
    lo = p + 1;
  }
  return lower_bound_key(key, lo, hi, x);
}

// smallest index with a nonzero mark in this block, and whether any candidate
// was deferred: one atomic each per block
__device__ __forceinline__ void block_first(int64_t first, bool deferred, unsigned long long* __restrict__ first_slot,
                                            unsigned* __restrict__ need) {
  __shared__ unsigned long long wmin[32];
  __shared__ int wdef[32];
  unsigned long long f = (unsigned long long)first;
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_down_sync(0xffffffffu, f, o);
    f = t < f ? t : f;
  }
  const int d = __any_sync(0xffffffffu, deferred) ? 1 : 0;
  if ((threadIdx.x & 31) == 0) {
    wmin[threadIdx.x >> 5] = f;
    wdef[threadIdx.x >> 5] = d;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = ~0ull;
    int any = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      m = wmin[w] < m ? wmin[w] : m;
      any |= wdef[w];
    }
    if (m != ~0ull) atomicMin(first_slot, m);
    if (any) atomicOr(need, 1u);
  }
}

// kPrefix false: the first pass over every particle (geometric criterion with
// the member filter): candidates whose cells at the levels that can merge hold
// at most kDirect particles are decided from direct sums, the others deferred.
// kPrefix true (only when something was deferred, or without the filter):
// the deferred particles (every particle without the filter) are decided from
// the prefix sums.
template <bool kPrefix>
__global__ void k_merge_mark(const int32_t* __restrict__ d_n, int64_t cap, const uint64_t* __restrict__ key,
                             const uint32_t* __restrict__ u, const uint32_t* __restrict__ kk,
                             const uint64_t* __restrict__ pre, int32_t* __restrict__ mend,
                             int32_t* __restrict__ keep, MergeParams mp, unsigned long long* __restrict__ first_slot,
                             unsigned* __restrict__ need) {
  if (kPrefix && !*need) return;
  const int64_t n = *d_n;
  const uint64_t* PK = pre;
  const uint64_t* PS = pre + (cap + 1);
  double rhs = 0.0;  // alpha a_min (dynamical)
  if (mp.criterion == DZS_CRIT_DYNAMICAL) {
    uint64_t c = *mp.amin2_slot;
    double amin2 = c ? __longlong_as_double((long long)~c) : __longlong_as_double(0x7ff0000000000000ll);
    rhs = __dmul_rn(mp.alpha, __dsqrt_rn(amin2));
  }
  int64_t first = INT64_MAX;
  bool deferred_any = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (kPrefix && mp.filter && mend[i] != kDeferred) continue;
    int32_t res = 0;
    bool deferred = false;
    bool cand = true;
    if (mp.filter) cand = dist2_obs(u[i], u[cap + i], u[2 * cap + i]) > mp.rb2;
    if (cand) {
      uint64_t ki = key[i];
      // candidate cells start at depth jstart: its bounds by galloping out
      // from i (the coarser cells only contain it), deeper ones inside the
      // previous
      const int j0 = mp.jstart;
      int64_t lo = 0, hi = n;
      for (int j = j0; j <= kMaxLevel; ++j) {
        int sh = 3 * (kMaxLevel - j);
        uint64_t cell = (ki >> sh) << sh;
        int64_t s, e;
        if (j == j0) {
          s = gallop_down(key, i, cell);
          e = gallop_up(key, i + 1, n, cell + (1ull << sh));
        } else {
          s = lower_bound_key(key, lo, i + 1, cell);
          e = lower_bound_key(key, i + 1, hi, cell + (1ull << sh));
        }
        lo = s;
        hi = e;
        if (e - s < 2) break;  // no finer cell holds two particles
        if (mp.criterion == DZS_CRIT_GEOMETRIC && mp.thr[j] == ~0ull) continue;
        uint64_t K = 0, S[3] = {0, 0, 0};
        if (kPrefix) {
          K = PK[e] - PK[s];
          for (int ax = 0; ax < 3; ++ax)
            S[ax] = PS[(int64_t)ax * (cap + 1) + e] - PS[(int64_t)ax * (cap + 1) + s];
        } else {
          if (e - s > kDirect) {
            deferred = true;
            break;
          }
          for (int64_t t = s; t < e; ++t) {
            const uint64_t m = kk[t];
            K += m;
            for (int ax = 0; ax < 3; ++ax) S[ax] += m * u[ax * cap + t];
          }
        }
        uint64_t d2 = 0;
        for (int ax = 0; ax < 3; ++ax) {
          uint32_t com = (uint32_t)((2 * S[ax] + K) / (2 * K));
          int64_t off = (int32_t)(com - 0x80000000u);
          d2 += (uint64_t)(off * off);
        }
        bool merge;
        if (mp.criterion == DZS_CRIT_DYNAMICAL) {
          merge = dynamical_merge(mp, d2, K, j, rhs);
        } else {
          uint64_t T = mp.thr[j];
          merge = d2 > T * T;
        }
        if (merge) {
          res = (s == i) ? (int32_t)e : -1;
          break;
        }
      }
    }
    mend[i] = deferred ? kDeferred : res;
    keep[i] = res >= 0 ? 1 : 0;
    if (res != 0 && i < first) first = i;
    deferred_any = deferred_any || deferred;
  }
  block_first(first, deferred_any, first_slot, need);
}

// the compacted state from the first changed particle on, into the spare
// arrays (rank = exclusive scan of keep); merged cells summed directly
template <class R>
__global__ void k_merge_write(const int32_t* __restrict__ d_n, int64_t cap, const int32_t* __restrict__ mend,
                              const int32_t* __restrict__ rank, const uint64_t* __restrict__ key,
                              const uint32_t* __restrict__ u, const R* __restrict__ p,
                              const uint32_t* __restrict__ k, const uint32_t* __restrict__ id,
                              const uint8_t* __restrict__ fl, const unsigned long long* __restrict__ first_slot,
                              uint64_t* __restrict__ key2, uint32_t* __restrict__ u2, R* __restrict__ p2,
                              uint32_t* __restrict__ k2, uint32_t* __restrict__ id2, uint8_t* __restrict__ fl2,
                              int32_t* __restrict__ d_n_out) {
  const int64_t n = *d_n;
  const int64_t first = *first_slot < (unsigned long long)n ? (int64_t)*first_slot : n;
  for (int64_t i = first + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t m = mend[i];
    if (m < 0) continue;
    int64_t j = rank[i];
    if (m == 0) {
      for (int ax = 0; ax < 3; ++ax) {
        u2[ax * cap + j] = u[ax * cap + i];
        p2[ax * cap + j] = p[ax * cap + i];
      }
      key2[j] = key[i];
      k2[j] = k[i];
      id2[j] = id[i];
      fl2[j] = fl[i];
      continue;
    }
    int64_t e = m;
    uint64_t K = 0;
    for (int64_t t = i; t < e; ++t) K += k[t];
    uint32_t com[3];
    for (int ax = 0; ax < 3; ++ax) {
      uint64_t S = 0;
      double acc = 0.0;  // left-to-right FP64 sum, no contraction
      for (int64_t t = i; t < e; ++t) {
        S += (uint64_t)k[t] * u[ax * cap + t];
        acc = __dadd_rn(acc, __dmul_rn((double)k[t], (double)p[ax * cap + t]));
      }
      com[ax] = (uint32_t)((2 * S + K) / (2 * K));
      u2[ax * cap + j] = com[ax];
      p2[ax * cap + j] = (R)(acc / (double)K);
    }
    uint32_t idm = id[i];
    for (int64_t t = i + 1; t < e; ++t) idm = min(idm, id[t]);
    key2[j] = morton_key(com[0], com[1], com[2]);
    k2[j] = (uint32_t)K;
    id2[j] = idm;
    fl2[j] = (uint8_t)(kFlMerged | kFlCrossed);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *d_n_out = rank[n];
}

// the changed tail [first, n_new) back into the state arrays
template <class R>
__global__ void k_merge_copyback(const int32_t* __restrict__ d_n_new, int64_t cap,
                                 const unsigned long long* __restrict__ first_slot, const uint64_t* __restrict__ key2,
                                 const uint32_t* __restrict__ u2, const R* __restrict__ p2,
                                 const uint32_t* __restrict__ k2, const uint32_t* __restrict__ id2,
                                 const uint8_t* __restrict__ fl2, uint64_t* __restrict__ key, uint32_t* __restrict__ u,
                                 R* __restrict__ p, uint32_t* __restrict__ k, uint32_t* __restrict__ id,
                                 uint8_t* __restrict__ fl) {
  const int64_t n = *d_n_new;
  const int64_t first = *first_slot < (unsigned long long)n ? (int64_t)*first_slot : n;
  for (int64_t i = first + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int ax = 0; ax < 3; ++ax) {
      u[ax * cap + i] = u2[ax * cap + i];
      p[ax * cap + i] = p2[ax * cap + i];
    }
    key[i] = key2[i];
    k[i] = k2[i];
    id[i] = id2[i];
    fl[i] = fl2[i];
  }
}

}  // namespace

void launch_mass_prefix(dzs_ctx* c) {
  c->launches += 3;
  Buffers& B = c->B;
  const int nchunks = (int)((c->cap + kChunk) / kChunk);
  uint64_t* tot = (uint64_t*)B.blocksum;
  k_prefix_totals<<<nchunks, 256, 0, c->stream>>>(B.n, c->cap, B.u, B.k, tot, nullptr);
  k_prefix_scan_totals<<<4, 1024, 0, c->stream>>>(tot, nchunks, nullptr);
  k_prefix_apply<<<nchunks, 256, 0, c->stream>>>(B.n, c->cap, B.u, B.k, tot, nchunks, B.prefix, nullptr);
}

void launch_amin2(dzs_ctx* c) {
  c->launches += 1;
  Buffers& B = c->B;
  unsigned long long* slot = (unsigned long long*)(B.counters + 14);
  cudaMemsetAsync(slot, 0, sizeof(uint64_t), c->stream);
  int grid = grid_for(c->N0);
  if (c->fp64)
    k_amin2<double><<<grid, kThreads, 0, c->stream>>>(B.n, c->cap, (const double*)B.g, B.fl, slot);
  else
    k_amin2<float><<<grid, kThreads, 0, c->stream>>>(B.n, c->cap, (const float*)B.g, B.fl, slot);
  c->amin2_ready = true;
}

// the dynamical criterion reads a_min^2 from counters[14] (launch_amin2 first)
void launch_merge(dzs_ctx* c, uint64_t rlat) {
  const bool dyn = c->P.dzs_criterion == DZS_CRIT_DYNAMICAL;
  Buffers& B = c->B;
  MergeParams mp;
  // a COM offset from the observer is below 2^31 per axis: d^2 <= 3 * 2^62,
  // so a level with T_j^2 >= 3 * 2^62 never merges
  const uint64_t d2max = 3ull << 62;
  for (int j = 0; j <= kMaxLevel; ++j) {
    uint64_t t = (c->merge_thr[j] == ~0ull) ? ~0ull : rlat + c->merge_thr[j];
    if (t != ~0ull && (t >= 4294967296ull || t * t >= d2max)) t = ~0ull;
    mp.thr[j] = t;
  }
  uint64_t rb = rlat + c->blat;
  mp.rb2 = (rb >= 4294967296ull) ? ~0ull : rb * rb;
  mp.jmin = c->jmin;
  mp.jstart = c->jmin > 1 ? c->jmin : 1;
  if (!dyn)
    while (mp.jstart <= kMaxLevel && mp.thr[mp.jstart] == ~0ull) ++mp.jstart;
  mp.filter = (!dyn && c->P.theta_dzs <= 0.5773502691896257) ? 1 : 0;
  mp.criterion = c->P.dzs_criterion;
  mp.rb = (double)rb;
  mp.scale = c->scale;
  mp.gm0 = c->gm0;
  mp.alpha = c->P.alpha_dyn;
  for (int j = 0; j <= kMaxLevel; ++j) {
    double l = std::ldexp(c->P.box, -j);
    mp.l2[j] = l * l;
  }
  uint64_t* slot = c->B.counters + 14;
  mp.amin2_slot = slot;
  unsigned long long* first = (unsigned long long*)(c->B.counters + 22);
  unsigned* need = (unsigned*)(c->B.counters + 23);
  cudaMemsetAsync(first, 0xff, sizeof(uint64_t), c->stream);
  int nchunks = (int)((c->cap + kChunk) / kChunk);
  uint64_t* tot = (uint64_t*)B.blocksum;
  int32_t* keep = B.iscan + (c->cap + 1);
  int32_t* rank = B.iscan;
  int grid = grid_for(c->N0);
  if (mp.filter) {
    c->launches += 1;
    cudaMemsetAsync(need, 0, sizeof(unsigned), c->stream);
    k_merge_mark<false><<<grid, kThreads, 0, c->stream>>>(B.n, c->cap, B.key, B.u, B.k, B.prefix, B.mend, keep, mp,
                                                          first, need);
  } else {
    cudaMemsetAsync(need, 1, sizeof(unsigned), c->stream);  // nonzero: every particle takes the prefix pass
  }
  // prefix sums and the second mark pass: they return at once unless needed
  c->launches += 4;
  k_prefix_totals<<<nchunks, 256, 0, c->stream>>>(B.n, c->cap, B.u, B.k, tot, need);
  k_prefix_scan_totals<<<4, 1024, 0, c->stream>>>(tot, nchunks, need);
  k_prefix_apply<<<nchunks, 256, 0, c->stream>>>(B.n, c->cap, B.u, B.k, tot, nchunks, B.prefix, need);
  k_merge_mark<true><<<grid, kThreads, 0, c->stream>>>(B.n, c->cap, B.key, B.u, B.k, B.prefix, B.mend, keep, mp,
                                                       first, need);
  c->launches += 5;
  exclusive_scan_i32(c, keep, rank, B.n, c->cap);
  if (c->fp64) {
    k_merge_write<double><<<grid, kThreads, 0, c->stream>>>(
        B.n, c->cap, B.mend, rank, B.key, B.u, (const double*)B.p, B.k, B.id, B.fl, first, B.key2, B.u2,
        (double*)B.p2, B.k2, B.id2, B.fl2, B.n + 1);
    k_merge_copyback<double><<<grid, kThreads, 0, c->stream>>>(B.n + 1, c->cap, first, B.key2, B.u2,
                                                               (const double*)B.p2, B.k2, B.id2, B.fl2, B.key, B.u,
                                                               (double*)B.p, B.k, B.id, B.fl);
  } else {
    k_merge_write<float><<<grid, kThreads, 0, c->stream>>>(
        B.n, c->cap, B.mend, rank, B.key, B.u, (const float*)B.p, B.k, B.id, B.fl, first, B.key2, B.u2,
        (float*)B.p2, B.k2, B.id2, B.fl2, B.n + 1);
    k_merge_copyback<float><<<grid, kThreads, 0, c->stream>>>(B.n + 1, c->cap, first, B.key2, B.u2,
                                                              (const float*)B.p2, B.k2, B.id2, B.fl2, B.key, B.u,
                                                              (float*)B.p, B.k, B.id, B.fl);
  }
  // new count staged in n[1] (every thread of the write kernel read n[0])
  cudaMemcpyAsync(B.n, B.n + 1, sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream);
}

}  // namespace dzs
