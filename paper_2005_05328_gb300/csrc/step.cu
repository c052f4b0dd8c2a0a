// step.cu -- opening kick + drift on the lattice + lightcone crossing test +
// Morton key (one fused pass), the compaction of crossing records into the
// lightcone ring, and the conservation diagnostics.
//
// Paper: global steps (Sec. 2.1); particles are written to the lightcone
// output as its boundary R_lc(a) meets them (Sec. 1 footnote, Sec. 3.1.3).
// A particle not yet flagged is recorded when d_n < R_lc(a_n) and
// d_n+1 >= R_lc(a_n+1), decided exactly on the integer lattice.
#include "common.cuh"
#include "observe.cuh"

namespace dzs {
namespace {

__device__ __forceinline__ float kicked(float p, float g, float k) { return fmaf(g, k, p); }
__device__ __forceinline__ double kicked(double p, double g, double k) { return fma(g, k, p); }

// p += g K1; u += rint(p D 2^32 / L); crossing; key.  Grid-stride over n.
// kDry: the same kick, drift and crossing test, nothing written; the number of
// particles that would cross is added to *count (the lightcone ring's room is
// checked with it before a step that might overflow a small ring)
template <class R, bool kDry>
__global__ void k_kick_drift(const int32_t* __restrict__ d_n, int64_t cap, uint32_t* __restrict__ u,
                             R* __restrict__ p, const R* __restrict__ g, uint8_t* __restrict__ fl,
                             uint64_t* __restrict__ key, int32_t* __restrict__ now, R kick,
                             double dlat, uint64_t r20, uint64_t r21, unsigned long long* __restrict__ count) {
  const int64_t n = *d_n;
  unsigned ncross = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t ub[3], ua[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const R pj = kicked(p[ax * cap + i], g[ax * cap + i], kick);
      if (!kDry) p[ax * cap + i] = pj;
      ub[ax] = u[ax * cap + i];
      long long du = __double2ll_rn((double)pj * dlat);
      ua[ax] = ub[ax] + (uint32_t)(unsigned long long)du;
      if (!kDry) u[ax * cap + i] = ua[ax];
    }
    uint8_t f = fl[i] & (uint8_t)~kFlNow;
    int32_t crossed = 0;
    if (!(f & kFlCrossed)) {
      uint64_t db = dist2_obs(ub[0], ub[1], ub[2]);
      uint64_t da = dist2_obs(ua[0], ua[1], ua[2]);
      if (db < r20 && da >= r21) {
        f |= (uint8_t)(kFlCrossed | kFlNow);
        crossed = 1;
      }
    }
    if (kDry) {
      ncross += (unsigned)crossed;
    } else {
      fl[i] = f;
      now[i] = crossed;
      key[i] = morton_key(ua[0], ua[1], ua[2]);
    }
  }
  if (kDry) {
    for (int o = 16; o > 0; o >>= 1) ncross += __shfl_down_sync(0xffffffffu, ncross, o);
    if ((threadIdx.x & 31) == 0 && ncross) atomicAdd(count, (unsigned long long)ncross);
  }
}

// one record per particle with the kFlNow bit, at ring slot head + rank
template <class R>
__global__ void k_records(const int32_t* __restrict__ d_n, int64_t cap, const uint32_t* __restrict__ u,
                          const R* __restrict__ p, const uint32_t* __restrict__ k,
                          const uint32_t* __restrict__ id, const uint8_t* __restrict__ fl,
                          const int32_t* __restrict__ rank, dzs_lc_record* __restrict__ ring,
                          uint64_t ring_cap, uint64_t* __restrict__ counters, uint64_t drained,
                          uint32_t* __restrict__ err, double dlat, double scale, double box,
                          double a0, double a1, double rlc0, double rlc1, ObserveTarget obs) {
  const int64_t n = *d_n;
  const uint64_t head = counters[0];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (!(fl[i] & kFlNow)) continue;
    uint64_t slot = head + (uint64_t)rank[i];
    const bool room = slot - drained < ring_cap;
    if (!room) atomicOr(err, kErrRing);
    if (!room && !obs.sky && !obs.grid) continue;
    uint32_t ua[3], ub[3];
    double pd[3];
    for (int ax = 0; ax < 3; ++ax) {
      ua[ax] = u[ax * cap + i];
      pd[ax] = (double)p[ax * cap + i];
      long long du = __double2ll_rn(pd[ax] * dlat);
      ub[ax] = ua[ax] - (uint32_t)(unsigned long long)du;
    }
    double sb = sqrt((double)dist2_obs(ub[0], ub[1], ub[2])) * scale - rlc0;
    double sa = sqrt((double)dist2_obs(ua[0], ua[1], ua[2])) * scale - rlc1;
    double t = sb / (sb - sa);
    if (!(t >= 0.0)) t = 0.0;
    if (t > 1.0) t = 1.0;
    dzs_lc_record r;
    r.id = id[i];
    r.k = k[i];
    r.a_cross = a0 + t * (a1 - a0);
    for (int ax = 0; ax < 3; ++ax) {
      double x = (double)ub[ax] * scale + t * (double)(int32_t)(ua[ax] - ub[ax]) * scale;
      if (x < 0.0) x += box;
      if (x >= box) x -= box;
      r.x[ax] = x;
      r.p[ax] = pd[ax];
    }
    observe_record(obs, r.k, r.a_cross, r.x);  // sky map / 3D lightcone, also for a dropped record
    if (room) ring[slot % ring_cap] = r;
  }
}

__global__ void k_records_advance(const int32_t* __restrict__ d_n, const int32_t* __restrict__ rank,
                                  uint64_t* __restrict__ counters, uint64_t ring_cap, uint64_t drained) {
  uint64_t total = (uint64_t)rank[*d_n];
  uint64_t head = counters[0];
  uint64_t room = ring_cap - (head - drained);
  if (total > room) {
    counters[1] += total - room;  // dropped
    total = room;
  }
  counters[0] = head + total;
}

// ---- diagnostics: exact integer sums by atomics, FP64 momentum by fixed-order
// block partials reduced by one block in block order
constexpr int kDiagBlocks = 304;

template <class R>
__global__ void k_diag_partial(const int32_t* __restrict__ d_n, int64_t cap, const uint32_t* __restrict__ u,
                               const R* __restrict__ p, const uint32_t* __restrict__ k,
                               double* __restrict__ part, unsigned long long* __restrict__ isum) {
  const int64_t n = *d_n;
  double s[3] = {0, 0, 0};
  unsigned long long ks = 0, us[3] = {0, 0, 0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t kk = k[i];
    ks += kk;
    for (int ax = 0; ax < 3; ++ax) {
      s[ax] += (double)kk * (double)p[ax * cap + i];
      us[ax] += (unsigned long long)kk * u[ax * cap + i];
    }
  }
  __shared__ double sh[3][kThreads];
  __shared__ unsigned long long ish[4][kThreads / 32];
  for (int ax = 0; ax < 3; ++ax) sh[ax][threadIdx.x] = s[ax];
  // integer sums: warp shuffles, then one atomic per block and sum (exact in
  // any order; an atomic per thread serialised on four addresses)
  for (int o = 16; o > 0; o >>= 1) {
    ks += __shfl_down_sync(0xffffffffu, ks, o);
    for (int ax = 0; ax < 3; ++ax) us[ax] += __shfl_down_sync(0xffffffffu, us[ax], o);
  }
  if ((threadIdx.x & 31) == 0) {
    ish[0][threadIdx.x >> 5] = ks;
    for (int ax = 0; ax < 3; ++ax) ish[1 + ax][threadIdx.x >> 5] = us[ax];
  }
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int ax = 0; ax < 3; ++ax) sh[ax][threadIdx.x] += sh[ax][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int ax = 0; ax < 3; ++ax) part[ax * kDiagBlocks + blockIdx.x] = sh[ax][0];
  if (threadIdx.x < 4) {
    unsigned long long t = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += ish[threadIdx.x][q];
    atomicAdd(&isum[threadIdx.x], t);
  }
}

// one warp per axis: lane-strided sums of the block partials, then a fixed
// shuffle tree (the same order every call)
__global__ void k_diag_final(const int32_t* __restrict__ d_n, const double* __restrict__ part,
                             const unsigned long long* __restrict__ isum, double* __restrict__ out,
                             double scale) {
  const int ax = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (ax >= 3) return;
  double s = 0;
  for (int b = lane; b < kDiagBlocks; b += 32) s += part[ax * kDiagBlocks + b];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) {
    out[1 + ax] = s;
    out[4 + ax] = (double)isum[1 + ax] * scale;
    if (ax == 0) {
      out[0] = (double)isum[0];
      out[7] = (double)*d_n;
    }
  }
}

template <class S, class D>
__global__ void k_convert(const S* __restrict__ src, D* __restrict__ dst, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (D)src[i];
}

}  // namespace

void launch_kick_drift(dzs_ctx* c, int step, bool, bool) {
  c->launches += 1;
  uint64_t r0 = c->T.rlat[step], r1 = c->T.rlat[step + 1];
  double dlat = c->T.drift[step] * c->lat;
  int grid = grid_for(c->N0);
  int32_t* now = c->B.iscan + (c->cap + 1);  // second half of the int scratch
  if (c->fp64)
    k_kick_drift<double, false><<<grid, kThreads, 0, c->stream>>>(c->B.n, c->cap, c->B.u, (double*)c->B.p,
                                                                  (const double*)c->B.g, c->B.fl, c->B.key, now,
                                                                  c->T.kick1[step], dlat, r0 * r0, r1 * r1, nullptr);
  else
    k_kick_drift<float, false><<<grid, kThreads, 0, c->stream>>>(c->B.n, c->cap, c->B.u, (float*)c->B.p,
                                                                 (const float*)c->B.g, c->B.fl, c->B.key, now,
                                                                 (float)c->T.kick1[step], dlat, r0 * r0, r1 * r1,
                                                                 nullptr);
}

// the number of particles that step `step` would record (a dry run of its
// kick, drift and crossing test), added to *count on the device
void launch_count_crossings(dzs_ctx* c, int step, unsigned long long* count) {
  c->launches += 1;
  uint64_t r0 = c->T.rlat[step], r1 = c->T.rlat[step + 1];
  double dlat = c->T.drift[step] * c->lat;
  int grid = grid_for(c->N0);
  if (c->fp64)
    k_kick_drift<double, true><<<grid, kThreads, 0, c->stream>>>(c->B.n, c->cap, c->B.u, (double*)c->B.p,
                                                                 (const double*)c->B.g, c->B.fl, nullptr, nullptr,
                                                                 c->T.kick1[step], dlat, r0 * r0, r1 * r1, count);
  else
    k_kick_drift<float, true><<<grid, kThreads, 0, c->stream>>>(c->B.n, c->cap, c->B.u, (float*)c->B.p,
                                                                (const float*)c->B.g, c->B.fl, nullptr, nullptr,
                                                                (float)c->T.kick1[step], dlat, r0 * r0, r1 * r1,
                                                                count);
}

void launch_records(dzs_ctx* c, int step) {
  c->launches += 5;
  int32_t* now = c->B.iscan + (c->cap + 1);
  int32_t* rank = c->B.iscan;
  exclusive_scan_i32(c, now, rank, c->B.n, c->cap);
  int grid = grid_for(c->N0);
  double dlat = c->T.drift[step] * c->lat;
  if (c->fp64)
    k_records<double><<<grid, kThreads, 0, c->stream>>>(
        c->B.n, c->cap, c->B.u, (const double*)c->B.p, c->B.k, c->B.id, c->B.fl, rank, c->B.ring,
        c->ring_cap, c->B.counters, c->drained, c->B.err, dlat, c->scale, c->P.box, c->T.a[step],
        c->T.a[step + 1], c->T.rlc[step], c->T.rlc[step + 1], c->obs);
  else
    k_records<float><<<grid, kThreads, 0, c->stream>>>(
        c->B.n, c->cap, c->B.u, (const float*)c->B.p, c->B.k, c->B.id, c->B.fl, rank, c->B.ring,
        c->ring_cap, c->B.counters, c->drained, c->B.err, dlat, c->scale, c->P.box, c->T.a[step],
        c->T.a[step + 1], c->T.rlc[step], c->T.rlc[step + 1], c->obs);
  k_records_advance<<<1, 1, 0, c->stream>>>(c->B.n, rank, c->B.counters, c->ring_cap, c->drained);
}

void launch_diagnostics(dzs_ctx* c) {
  c->launches += 2;
  double* part = c->B.diag + 8;
  unsigned long long* isum = (unsigned long long*)(c->B.counters + 8);
  cudaMemsetAsync(isum, 0, 4 * sizeof(unsigned long long), c->stream);
  if (c->fp64)
    k_diag_partial<double><<<kDiagBlocks, kThreads, 0, c->stream>>>(c->B.n, c->cap, c->B.u,
                                                                    (const double*)c->B.p, c->B.k, part, isum);
  else
    k_diag_partial<float><<<kDiagBlocks, kThreads, 0, c->stream>>>(c->B.n, c->cap, c->B.u,
                                                                   (const float*)c->B.p, c->B.k, part, isum);
  k_diag_final<<<1, 96, 0, c->stream>>>(c->B.n, part, isum, c->B.diag, c->scale);
}

void launch_to_double(dzs_ctx* c, const void* src, int64_t count, double* dst) {
  if (c->fp64)
    cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  else
    k_convert<float, double><<<grid_for(count), kThreads, 0, c->stream>>>((const float*)src, dst, count);
}

void launch_from_double(dzs_ctx* c, const double* src, int64_t count, void* dst) {
  if (c->fp64)
    cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  else
    k_convert<double, float><<<grid_for(count), kThreads, 0, c->stream>>>(src, (float*)dst, count);
}

}  // namespace dzs
