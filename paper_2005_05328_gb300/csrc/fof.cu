// fof.cu -- friends-of-friends haloes on the GPU (paper Sec. 3.1.1: the
// lightcone halo mass function is built from FoF catalogues of frequent
// outputs, keeping the haloes entirely inside the lightcone).
//
// Friends: minimum-image lattice distance d^2 <= T, T = floor((link 2^32 /
// n1d)^2) (link in units of the initial mean spacing).  On the Morton-sorted
// particles, cells of a depth whose side is at least the linking length are
// contiguous runs (CSR table); each particle scans the 27 neighbour cells and
// unites itself with every later friend.  Union-find without locks: a root is
// only ever hooked under a smaller index (one compare-and-swap; a failed swap
// means another thread changed that root, so the union retries with the new
// roots), so every component ends with its smallest sorted index as root,
// whatever the schedule.  Per component, exact integer sums: count, mass,
// mass-weighted offsets from the member with the smallest caller-order index
// (the halo's label), the largest squared distance from the observer.
#include "common.cuh"

namespace dzs {
namespace {

constexpr int kUnionTries = 1 << 20;  // a union gives up (error bit) after this many retries

__device__ __forceinline__ int32_t uf_find(const int32_t* par, int32_t x) {
  // parents only ever decrease, so the chain ends at the root
  int32_t p = ((volatile const int32_t*)par)[x];
  while (p != x) {
    x = p;
    p = ((volatile const int32_t*)par)[x];
  }
  return x;
}

__device__ __forceinline__ void uf_union(int32_t* par, int32_t a, int32_t b, uint32_t* err) {
  for (int t = 0; t < kUnionTries; ++t) {
    a = uf_find(par, a);
    b = uf_find(par, b);
    if (a == b) return;
    if (a > b) {
      const int32_t s = a;
      a = b;
      b = s;
    }
    if (atomicCAS(&par[b], b, a) == b) return;
  }
  atomicOr(err, kErrGroups);
}

__global__ void k_fof_init(const int32_t* __restrict__ d_n, int32_t* __restrict__ par, int32_t* __restrict__ cnt,
                           unsigned long long* __restrict__ mass, unsigned long long* __restrict__ rmax2,
                           int32_t* __restrict__ first, const uint32_t* __restrict__ idx, int32_t* __restrict__ inv,
                           unsigned long long* __restrict__ S) {
  const int64_t n = *d_n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    par[i] = (int32_t)i;
    cnt[i] = 0;
    mass[i] = 0;
    rmax2[i] = 0;
    first[i] = 0x7fffffff;
    inv[idx[i]] = (int32_t)i;  // caller order -> sorted position
    S[i] = S[n + i] = S[2 * n + i] = 0;
  }
}

__global__ void k_fof_link(const int32_t* __restrict__ d_n, int64_t cap, const uint32_t* __restrict__ u,
                           const int32_t* __restrict__ start, int depth, uint64_t T, int32_t* __restrict__ par,
                           uint32_t* __restrict__ err) {
  const int64_t n = *d_n;
  const int sh = 32 - depth;
  const uint32_t mask = (1u << depth) - 1u;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t xi = u[i], yi = u[cap + i], zi = u[2 * cap + i];
    const uint32_t cx = xi >> sh, cy = yi >> sh, cz = zi >> sh;
    for (int o = 0; o < 27; ++o) {
      const uint32_t ax = (cx + (uint32_t)(o / 9) - 1u) & mask, ay = (cy + (uint32_t)((o / 3) % 3) - 1u) & mask,
                     az = (cz + (uint32_t)(o % 3) - 1u) & mask;
      const uint64_t c = (spread3(ax) << 2) | (spread3(ay) << 1) | spread3(az);
      const int32_t s = start[c], e = start[c + 1];
      for (int32_t j = s > (int32_t)i + 1 ? s : (int32_t)i + 1; j < e; ++j) {
        const int64_t dx = (int32_t)(u[j] - xi), dy = (int32_t)(u[cap + j] - yi), dz = (int32_t)(u[2 * cap + j] - zi);
        const uint64_t d2 = (uint64_t)(dx * dx) + (uint64_t)(dy * dy) + (uint64_t)(dz * dz);
        if (d2 <= T) uf_union(par, (int32_t)i, j, err);
      }
    }
  }
}

// roots, sizes, masses, the observer distance bound and the label (smallest
// caller-order index) of every component
__global__ void k_fof_roots(const int32_t* __restrict__ d_n, int64_t cap, const uint32_t* __restrict__ u,
                            const uint32_t* __restrict__ k, const uint32_t* __restrict__ idx,
                            int32_t* __restrict__ par, int32_t* __restrict__ cnt,
                            unsigned long long* __restrict__ mass, unsigned long long* __restrict__ rmax2,
                            int32_t* __restrict__ first) {
  const int64_t n = *d_n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = uf_find(par, (int32_t)i);
    atomicAdd(&cnt[r], 1);
    atomicAdd(&mass[r], (unsigned long long)k[i]);
    atomicMax(&rmax2[r], (unsigned long long)dist2_obs(u[i], u[cap + i], u[2 * cap + i]));
    atomicMin(&first[r], (int32_t)idx[i]);
  }
}

// label every particle with its root (full compression), then offsets from the
// labelling member
__global__ void k_fof_offsets(const int32_t* __restrict__ d_n, int64_t cap, const uint32_t* __restrict__ u,
                              const uint32_t* __restrict__ k, int32_t* __restrict__ par,
                              const int32_t* __restrict__ first, const int32_t* __restrict__ inv,
                              unsigned long long* __restrict__ S) {
  const int64_t n = *d_n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = uf_find(par, (int32_t)i);
    const int32_t f = inv[first[r]];  // sorted position of the labelling member
    const long long kk = (long long)k[i];
    atomicAdd(&S[r], (unsigned long long)(kk * (long long)(int32_t)(u[i] - u[f])));
    atomicAdd(&S[n + r], (unsigned long long)(kk * (long long)(int32_t)(u[cap + i] - u[cap + f])));
    atomicAdd(&S[2 * n + r], (unsigned long long)(kk * (long long)(int32_t)(u[2 * cap + i] - u[2 * cap + f])));
  }
}

__global__ void k_fof_flags(const int32_t* __restrict__ d_n, const int32_t* __restrict__ par,
                            const int32_t* __restrict__ cnt, int nmin, int32_t* __restrict__ flag) {
  const int64_t n = *d_n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = (par[i] == (int32_t)i && cnt[i] >= nmin) ? 1 : 0;
}

__global__ void k_fof_write(const int32_t* __restrict__ d_n, int64_t cap, const uint32_t* __restrict__ u,
                            const int32_t* __restrict__ par, const int32_t* __restrict__ cnt,
                            const unsigned long long* __restrict__ mass, const unsigned long long* __restrict__ rmax2,
                            const int32_t* __restrict__ first, const int32_t* __restrict__ inv,
                            const unsigned long long* __restrict__ S, const int32_t* __restrict__ rank, int nmin,
                            double scale, double box, dzs_halo* __restrict__ out, int32_t* __restrict__ nh) {
  const int64_t n = *d_n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (par[i] != (int32_t)i || cnt[i] < nmin) continue;
    dzs_halo h;
    h.first = first[i];
    h.count = cnt[i];
    h.mass = mass[i];
    h.rmax2 = rmax2[i];
    const int32_t f = inv[first[i]];
    const double K = (double)mass[i];
    for (int ax = 0; ax < 3; ++ax) {
      const double off = (double)(long long)S[ax * n + i];
      double x = __dmul_rn(__dadd_rn((double)u[ax * cap + f], __ddiv_rn(off, K)), scale);
      if (x < 0.0) x = __dadd_rn(x, box);
      if (x >= box) x = __dsub_rn(x, box);
      h.x[ax] = x;
    }
    out[rank[i]] = h;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *nh = rank[n];
}

__global__ void k_fof_labels(const int32_t* __restrict__ d_n, const int32_t* __restrict__ par,
                             const int32_t* __restrict__ cnt, const int32_t* __restrict__ first,
                             const uint32_t* __restrict__ idx, int nmin, int64_t* __restrict__ label) {
  const int64_t n = *d_n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = uf_find(par, (int32_t)i);
    label[idx[i]] = cnt[r] >= nmin ? (int64_t)first[r] : -1;
  }
}

__global__ void k_cell_table(const int32_t* __restrict__ d_n, const uint64_t* __restrict__ key, int sh,
                             int64_t ncell, int32_t* __restrict__ start) {
  const int64_t n = *d_n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t ci = (i < n) ? (int64_t)(key[i] >> sh) : ncell;
    int64_t cp = (i > 0) ? (int64_t)(key[i - 1] >> sh) : -1;
    for (int64_t q = cp + 1; q <= ci; ++q) start[q] = (int32_t)i;
  }
}

}  // namespace

// FoF on the (sorted) state with B.idx = the caller-order index of each sorted
// particle; scratch: prefix (per-root records), convert (offset sums), cicw
// (halo records, nmin >= 2 keeps them within 32 bytes per particle), the PM
// cell table (cells of depth `depth`).  Leaves the halo count in n[2].
void launch_fof(dzs_ctx* c, int depth, uint64_t T, int nmin, int64_t* d_label, dzs_halo** d_halos) {
  c->launches += 9;
  Buffers& B = c->B;
  const int64_t cap = c->cap;
  char* pre = (char*)B.prefix;
  unsigned long long* mass = (unsigned long long*)pre;
  unsigned long long* rmax2 = mass + cap;
  int32_t* par = (int32_t*)(rmax2 + cap);
  int32_t* cnt = par + cap;
  int32_t* first = cnt + cap;
  int32_t* inv = first + cap;
  unsigned long long* S = (unsigned long long*)B.convert;
  dzs_halo* out = (dzs_halo*)B.cicw;
  const int grid = grid_for(c->N0);
  const int64_t ncell = (int64_t)1 << (3 * depth);
  k_cell_table<<<grid_for(c->N0 + 1), kThreads, 0, c->stream>>>(B.n, B.key, 3 * (kMaxLevel - depth), ncell,
                                                                B.cell_start);
  k_fof_init<<<grid, kThreads, 0, c->stream>>>(B.n, par, cnt, mass, rmax2, first, B.idx, inv, S);
  k_fof_link<<<grid, kThreads, 0, c->stream>>>(B.n, cap, B.u, B.cell_start, depth, T, par, B.err);
  k_fof_roots<<<grid, kThreads, 0, c->stream>>>(B.n, cap, B.u, B.k, B.idx, par, cnt, mass, rmax2, first);
  k_fof_offsets<<<grid, kThreads, 0, c->stream>>>(B.n, cap, B.u, B.k, par, first, inv, S);
  int32_t* flag = B.iscan + (cap + 1);
  int32_t* rank = B.iscan;
  k_fof_flags<<<grid, kThreads, 0, c->stream>>>(B.n, par, cnt, nmin, flag);
  exclusive_scan_i32(c, flag, rank, B.n, cap);
  k_fof_write<<<grid, kThreads, 0, c->stream>>>(B.n, cap, B.u, par, cnt, mass, rmax2, first, inv, S, rank, nmin,
                                                c->scale, c->P.box, out, B.n + 2);
  if (d_label)
    k_fof_labels<<<grid, kThreads, 0, c->stream>>>(B.n, par, cnt, first, B.idx, nmin, d_label);
  *d_halos = out;
}

}  // namespace dzs
