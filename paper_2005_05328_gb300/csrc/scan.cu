// scan.cu -- deterministic exclusive prefix sum of int32 values whose count
// lives on the device (the particle count changes on the device when DZS
// merges).  Three launches: per-chunk totals, a single-block scan of the
// totals, per-chunk scans.  Integer sums: the result does not depend on the
// launch shape.  Used by record compaction, the merge compaction and the
// group list.
#include "common.cuh"

namespace dzs {
namespace {

constexpr int kChunk = 1024;  // items per block (256 threads x 4)

__device__ __forceinline__ int32_t warp_incl_scan(int32_t v) {
  const unsigned lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= (unsigned)o) v += t;
  }
  return v;
}

// block-wide exclusive scan of one value per thread; returns the block total
__device__ int32_t block_excl_scan(int32_t v, int32_t* excl) {
  __shared__ int32_t warp_off[32];
  __shared__ int32_t block_total;  // separate slot: a 1024-thread block uses all 32 offsets
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int32_t inc = warp_incl_scan(v);
  if (lane == 31) warp_off[w] = inc;
  __syncthreads();
  if (w == 0) {
    int32_t t = lane < nw ? warp_off[lane] : 0;
    int32_t ti = warp_incl_scan(t);
    if (lane < nw) warp_off[lane] = ti - t;
    if (lane == nw - 1) block_total = ti;
  }
  __syncthreads();
  *excl = inc - v + warp_off[w];
  int32_t total = block_total;
  __syncthreads();
  return total;
}

__global__ void k_chunk_totals(const int32_t* __restrict__ in, const int32_t* d_n,
                               int64_t* __restrict__ tot) {
  const int64_t n = *d_n;
  int64_t base = (int64_t)blockIdx.x * kChunk;
  int32_t s = 0;
  for (int t = threadIdx.x; t < kChunk; t += blockDim.x) {
    int64_t i = base + t;
    if (i < n) s += in[i];
  }
  int32_t ex;
  int32_t total = block_excl_scan(s, &ex);
  if (threadIdx.x == 0) tot[blockIdx.x] = total;
}

__global__ void k_scan_totals(int64_t* __restrict__ tot, int nchunks) {
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nchunks; base += blockDim.x) {
    int i = base + threadIdx.x;
    int32_t v = i < nchunks ? (int32_t)tot[i] : 0;
    int32_t ex;
    int32_t total = block_excl_scan(v, &ex);
    if (i < nchunks) tot[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) tot[nchunks] = carry;
}

// out[i] = sum_{j < i} in[j] for i <= n (out[n] = total)
__global__ void k_chunk_scan(const int32_t* __restrict__ in, const int32_t* d_n,
                             const int64_t* __restrict__ tot, int32_t* __restrict__ out,
                             int nchunks) {
  const int64_t n = *d_n;
  int64_t base = (int64_t)blockIdx.x * kChunk;
  if (base > n) return;
  // each thread owns 4 consecutive items
  int64_t i0 = base + 4 * threadIdx.x;
  int32_t v[4], s = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    v[q] = (i0 + q < n) ? in[i0 + q] : 0;
    s += v[q];
  }
  int32_t ex;
  block_excl_scan(s, &ex);
  int32_t run = (int32_t)tot[blockIdx.x] + ex;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (i0 + q <= n) out[i0 + q] = run;
    run += v[q];
  }
}

}  // namespace

void exclusive_scan_i32(dzs_ctx* c, const int32_t* in, int32_t* out, const int32_t* d_n, int64_t cap) {
  int nchunks = (int)((cap + kChunk) / kChunk);  // covers index cap itself
  k_chunk_totals<<<nchunks, 256, 0, c->stream>>>(in, d_n, c->B.blocksum);
  k_scan_totals<<<1, 1024, 0, c->stream>>>(c->B.blocksum, nchunks);
  k_chunk_scan<<<nchunks, 256, 0, c->stream>>>(in, d_n, c->B.blocksum, out, nchunks);
}

}  // namespace dzs
