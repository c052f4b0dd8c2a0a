// tree.cu -- oct-tree over the Morton-sorted particles (paper Sec. 2.1: root =
// box, nodes split into octants, nodes carry mass and centre of mass).
//
// Top-down, one launch per depth: a node with more than B particles (and depth
// < 21) finds its non-empty octants and appends them to the next depth with
// one atomic allocation.  Down to the PM mesh depth m (M = 2^m) the octant
// boundaries are read from the CSR table of the depth-m Morton cells (the PM
// deposit uses the same table), so the few huge nodes near the root cost O(1)
// instead of long chains of dependent binary-search loads; deeper nodes are
// small and search their keys.  Node numbering within a depth depends on
// scheduling, the tree structure does not: every consumer walks structure
// (children in octant order), so results are deterministic.  Bottom-up, in
// one launch: every leaf sums its particles, then climbs -- the last child to
// arrive at a parent (atomic counter) sums the children and goes on, the
// others stop; nothing waits.  Exact integer mass and mass-weighted position
// (uint64), the rounded integer COM and the largest member multiplicity (node
// softening).  Walk groups (node with <= G particles whose parent holds more,
// or a leaf) are listed in Morton order.
#include <cuda/atomic>

#include "common.cuh"

namespace dzs {
namespace {

__global__ void k_tree_root(const int32_t* __restrict__ d_n, Node* __restrict__ nodes, int32_t* __restrict__ lvl,
                            int32_t* __restrict__ group_head, int32_t* __restrict__ parent, int G) {
  int t = threadIdx.x;
  if (t < kMaxLevel + 2) lvl[t] = 0;
  if (t == 0) {
    parent[0] = -1;
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

__global__ void k_tree_down(int level, const uint64_t* __restrict__ key, const int32_t* __restrict__ cstart,
                            int depth_m, Node* __restrict__ nodes, int32_t* __restrict__ lvl,
                            int32_t* __restrict__ group_head, int32_t* __restrict__ parent,
                            int32_t* __restrict__ arrive, int64_t node_cap, int B, int G,
                            uint32_t* __restrict__ err) {
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
    if (level + 1 <= depth_m) {
      // child cell (pref | d) at depth level + 1 starts where its first
      // depth-m sub-cell starts
      const int dsh = 3 * (depth_m - (level + 1));
      for (int d = 1; d < 8; ++d) bnd[d] = cstart[(pref | (uint64_t)d) << dsh];
    } else {
      for (int d = 1; d < 8; ++d) bnd[d] = lb(key, bnd[d - 1], e, (pref | (uint64_t)d) << sh);
    }
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
      parent[first + q] = (int32_t)ni;
      bool leaf = c.count <= B || level + 1 == kMaxLevel;
      if (nd.count > G && (c.count <= G || leaf)) group_head[c.start] = (int32_t)(first + q);
      ++q;
    }
    nodes[ni].child = (int32_t)first;
    nodes[ni].meta = (uint32_t)level | ((uint32_t)nch << 8);
    arrive[ni] = 0;
  }
}

__device__ __forceinline__ void write_node_sums(Node* __restrict__ nodes, uint64_t* __restrict__ nsum,
                                                int64_t node_cap, int64_t ni, uint64_t K, const uint64_t (&S)[3],
                                                uint32_t kmax) {
  for (int ax = 0; ax < 3; ++ax) nsum[ax * node_cap + ni] = S[ax];
  nodes[ni].mass = (uint32_t)K;
  nodes[ni].kmax = kmax;
  if (K > 0) {
    nodes[ni].comx = (uint32_t)((2 * S[0] + K) / (2 * K));
    nodes[ni].comy = (uint32_t)((2 * S[1] + K) / (2 * K));
    nodes[ni].comz = (uint32_t)((2 * S[2] + K) / (2 * K));
  }
}

// all depths in one launch: leaves sum their particles and climb; at each
// parent the last child to arrive (after a fence on its writes) sums the
// children, read from L2 (the writers are other blocks), and climbs on
__global__ void k_tree_up_all(const int32_t* __restrict__ lvl, int64_t cap, const uint32_t* __restrict__ u,
                              const uint32_t* __restrict__ k, Node* __restrict__ nodes, uint64_t* __restrict__ nsum,
                              int64_t node_cap, const int32_t* __restrict__ parent, int32_t* __restrict__ arrive) {
  int64_t total = 0;
  for (int j = 0; j <= kMaxLevel; ++j) total += lvl[j];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const Node nd = nodes[t];
    if (nd.child >= 0) continue;  // finished by its last child
    uint64_t K = 0, S[3] = {0, 0, 0};
    uint32_t kmax = 0;
    for (int64_t i = nd.start; i < (int64_t)nd.start + nd.count; ++i) {
      uint32_t kk = k[i];
      K += kk;
      kmax = max(kmax, kk);
      for (int ax = 0; ax < 3; ++ax) S[ax] += (uint64_t)kk * u[ax * cap + i];
    }
    write_node_sums(nodes, nsum, node_cap, t, K, S, kmax);
    int64_t cur = t;
    for (;;) {
      const int32_t par = parent[cur];
      if (par < 0) break;
      const int nch = (int)((nodes[par].meta >> 8) & 0xff);
      // release this subtree's sums with the arrival; the last arriver acquires
      // every sibling's
      cuda::atomic_ref<int32_t, cuda::thread_scope_device> arr(arrive[par]);
      if (arr.fetch_add(1, cuda::memory_order_acq_rel) + 1 < nch) break;
      const int32_t c0 = nodes[par].child;
      uint64_t PK = 0, PS[3] = {0, 0, 0};
      uint32_t pkmax = 0;
      for (int q = 0; q < nch; ++q) {
        const int64_t ci = (int64_t)c0 + q;
        PK += __ldcg(&nodes[ci].mass);
        pkmax = max(pkmax, __ldcg(&nodes[ci].kmax));
        for (int ax = 0; ax < 3; ++ax) PS[ax] += __ldcg(&nsum[ax * node_cap + ci]);
      }
      write_node_sums(nodes, nsum, node_cap, par, PK, PS, pkmax);
      cur = par;
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
  c->launches += 28;
  Buffers& B = c->B;
  // the depth-m Morton cell table (also the PM deposit's)
  launch_cell_start(c);
  cudaMemsetAsync(B.group_head, 0xff, sizeof(int32_t) * c->cap, c->stream);
  k_tree_root<<<1, 32, 0, c->stream>>>(B.n, B.nodes, B.lvl_count, B.group_head, B.parent, c->P.walk_group);
  int grid = grid_for(c->N0, kThreads, 152 * 2);
  for (int j = 0; j < kMaxLevel; ++j)
    k_tree_down<<<grid, kThreads, 0, c->stream>>>(j, B.key, B.cell_start, c->logM, B.nodes, B.lvl_count,
                                                  B.group_head, B.parent, B.arrive, c->node_cap, c->P.leaf_bucket,
                                                  c->P.walk_group, B.err);
  k_tree_up_all<<<grid_for(c->node_cap, kThreads, 152 * 8), kThreads, 0, c->stream>>>(
      B.lvl_count, c->cap, B.u, B.k, B.nodes, B.nsum, c->node_cap, B.parent, B.arrive);
  int32_t* flag = B.iscan + (c->cap + 1);
  int32_t* rank = B.iscan;
  k_group_flags<<<grid_for(c->N0), kThreads, 0, c->stream>>>(B.n, B.group_head, flag);
  exclusive_scan_i32(c, flag, rank, B.n, c->cap);
  k_group_list<<<grid_for(c->N0), kThreads, 0, c->stream>>>(B.n, B.group_head, rank, B.groups, B.counters,
                                                            B.lvl_count);
}

}  // namespace dzs
