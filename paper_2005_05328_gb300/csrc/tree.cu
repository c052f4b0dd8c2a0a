// tree.cu -- oct-tree over the Morton-sorted particles (paper Sec. 2.1: root =
// box, nodes split into octants, nodes carry mass and centre of mass).
//
// Top-down, one launch per depth: a node with more than B particles (and depth
// < 21) finds its non-empty octants by binary search on the sorted keys and
// appends them to the next depth with one atomic allocation.  Node numbering
// within a depth depends on scheduling, the tree structure does not: every
// consumer walks structure (children in octant order), so results are
// deterministic.  Bottom-up, one launch per depth: exact integer mass and
// mass-weighted position (uint64), the rounded integer COM and the largest
// member multiplicity (node softening).  Walk groups (node with <= G
// particles whose parent holds more, or a leaf) are listed in Morton order.
#include "common.cuh"

namespace dzs {
namespace {

__global__ void k_tree_root(const int32_t* __restrict__ d_n, Node* __restrict__ nodes, int32_t* __restrict__ lvl,
                            int32_t* __restrict__ group_head, int G) {
  int t = threadIdx.x;
  if (t < kMaxLevel + 2) lvl[t] = 0;
  if (t == 0) {
    int32_t n = *d_n;
    Node r;
    r.cx = r.cy = r.cz = 0x80000000u;
    r.comx = r.comy = r.comz = 0x80000000u;
    r.mass = 0;
    r.kmax = 0;
    r.start = 0;
    r.count = n;
    r.child = -1;
    r.meta = 0;
    nodes[0] = r;
    lvl[0] = n > 0 ? 1 : 0;
    if (n > 0 && n <= G) group_head[0] = 0;
  }
}

__device__ __forceinline__ int64_t lb(const uint64_t* __restrict__ key, int64_t lo, int64_t hi, uint64_t x) {
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (key[mid] < x)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

__global__ void k_tree_down(int level, const uint64_t* __restrict__ key, Node* __restrict__ nodes,
                            int32_t* __restrict__ lvl, int32_t* __restrict__ group_head, int64_t node_cap,
                            int B, int G, uint32_t* __restrict__ err) {
  int64_t base = 0;
  for (int j = 0; j < level; ++j) base += lvl[j];
  const int64_t cnt = lvl[level];
  const int64_t child_base = base + cnt;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ni = base + t;
    Node nd = nodes[ni];
    if (nd.count <= B || level == kMaxLevel) continue;  // leaf
    const int64_t s = nd.start, e = (int64_t)nd.start + nd.count;
    const int sh = 3 * (kMaxLevel - (level + 1));
    const uint64_t pref = (key[s] >> (sh + 3)) << 3;  // parent prefix, shifted to child digit
    int64_t bnd[9];
    bnd[0] = s;
    bnd[8] = e;
    for (int d = 1; d < 8; ++d) bnd[d] = lb(key, bnd[d - 1], e, (pref | (uint64_t)d) << sh);
    int nch = 0;
    for (int d = 0; d < 8; ++d) nch += (bnd[d + 1] > bnd[d]) ? 1 : 0;
    int64_t off = atomicAdd(&lvl[level + 1], nch);
    int64_t first = child_base + off;
    if (first + nch > node_cap) {
      atomicOr(err, kErrNodes);
      continue;  // left as a leaf: the walk then sums its particles directly
    }
    const uint32_t lc = 1u << (31 - level);  // child side 2^(32 - level - 1)
    int q = 0;
    for (int d = 0; d < 8; ++d) {
      if (bnd[d + 1] == bnd[d]) continue;
      Node c;
      const uint32_t h = lc >> 1;
      c.cx = (d & 4) ? nd.cx + h : nd.cx - h;
      c.cy = (d & 2) ? nd.cy + h : nd.cy - h;
      c.cz = (d & 1) ? nd.cz + h : nd.cz - h;
      c.comx = c.comy = c.comz = 0;
      c.mass = 0;
      c.kmax = 0;
      c.start = (int32_t)bnd[d];
      c.count = (int32_t)(bnd[d + 1] - bnd[d]);
      c.child = -1;
      c.meta = (uint32_t)(level + 1);
      nodes[first + q] = c;
      bool leaf = c.count <= B || level + 1 == kMaxLevel;
      if (nd.count > G && (c.count <= G || leaf)) group_head[c.start] = (int32_t)(first + q);
      ++q;
    }
    nodes[ni].child = (int32_t)first;
    nodes[ni].meta = (uint32_t)level | ((uint32_t)nch << 8);
  }
}

__global__ void k_tree_up(int level, const int32_t* __restrict__ lvl, int64_t cap, const uint32_t* __restrict__ u,
                          const uint32_t* __restrict__ k, Node* __restrict__ nodes, uint64_t* __restrict__ nsum,
                          int64_t node_cap) {
  int64_t base = 0;
  for (int j = 0; j < level; ++j) base += lvl[j];
  const int64_t cnt = lvl[level];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ni = base + t;
    Node nd = nodes[ni];
    uint64_t K = 0, S[3] = {0, 0, 0};
    uint32_t kmax = 0;
    if (nd.child < 0) {
      for (int64_t i = nd.start; i < (int64_t)nd.start + nd.count; ++i) {
        uint32_t kk = k[i];
        K += kk;
        kmax = max(kmax, kk);
        for (int ax = 0; ax < 3; ++ax) S[ax] += (uint64_t)kk * u[ax * cap + i];
      }
    } else {
      int nch = (nd.meta >> 8) & 0xff;
      for (int q = 0; q < nch; ++q) {
        int64_t ci = nd.child + q;
        K += nodes[ci].mass;
        kmax = max(kmax, nodes[ci].kmax);
        for (int ax = 0; ax < 3; ++ax) S[ax] += nsum[ax * node_cap + ci];
      }
    }
    for (int ax = 0; ax < 3; ++ax) nsum[ax * node_cap + ni] = S[ax];
    nodes[ni].mass = (uint32_t)K;
    nodes[ni].kmax = kmax;
    if (K > 0) {
      nodes[ni].comx = (uint32_t)((2 * S[0] + K) / (2 * K));
      nodes[ni].comy = (uint32_t)((2 * S[1] + K) / (2 * K));
      nodes[ni].comz = (uint32_t)((2 * S[2] + K) / (2 * K));
    }
  }
}

__global__ void k_group_flags(const int32_t* __restrict__ d_n, const int32_t* __restrict__ head,
                              int32_t* __restrict__ flag) {
  const int64_t n = *d_n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = head[i] >= 0 ? 1 : 0;
}

__global__ void k_group_list(const int32_t* __restrict__ d_n, const int32_t* __restrict__ head,
                             const int32_t* __restrict__ rank, int32_t* __restrict__ groups,
                             uint64_t* __restrict__ counters, const int32_t* __restrict__ lvl) {
  const int64_t n = *d_n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (head[i] >= 0) groups[rank[i]] = head[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    counters[2] = (uint64_t)rank[n];
    uint64_t tot = 0;
    for (int j = 0; j <= kMaxLevel; ++j) tot += (uint64_t)lvl[j];
    counters[3] = tot;
  }
}

}  // namespace

void launch_tree(dzs_ctx* c) {
  c->launches += 49;
  Buffers& B = c->B;
  cudaMemsetAsync(B.group_head, 0xff, sizeof(int32_t) * c->cap, c->stream);
  k_tree_root<<<1, 32, 0, c->stream>>>(B.n, B.nodes, B.lvl_count, B.group_head, c->P.walk_group);
  int grid = grid_for(c->N0, kThreads, 152 * 8);
  for (int j = 0; j < kMaxLevel; ++j)
    k_tree_down<<<grid, kThreads, 0, c->stream>>>(j, B.key, B.nodes, B.lvl_count, B.group_head, c->node_cap,
                                                  c->P.leaf_bucket, c->P.walk_group, B.err);
  for (int j = kMaxLevel; j >= 0; --j)
    k_tree_up<<<grid, kThreads, 0, c->stream>>>(j, B.lvl_count, c->cap, B.u, B.k, B.nodes, B.nsum, c->node_cap);
  int32_t* flag = B.iscan + (c->cap + 1);
  int32_t* rank = B.iscan;
  k_group_flags<<<grid_for(c->N0), kThreads, 0, c->stream>>>(B.n, B.group_head, flag);
  exclusive_scan_i32(c, flag, rank, B.n, c->cap);
  k_group_list<<<grid_for(c->N0), kThreads, 0, c->stream>>>(B.n, B.group_head, rank, B.groups, B.counters,
                                                            B.lvl_count);
}

}  // namespace dzs
