// tree.cu -- oct-tree over the Morton-sorted particles (paper Sec. 2.1: root =
// box, nodes split into octants, nodes carry mass and centre of mass).
//
// The tree is the top-down one (a cell is split when it holds more than B
// particles and is above depth 21), built without a pass per depth.  Every
// node is a Morton cell and starts at a particle: the particle i that opens a
// cell at depth j (its key differs from key[i-1] within the first j octal
// digits, i.e. L_i < j with L_i the digits key[i-1] and key[i] share) owns
// that node exactly when the enclosing depth-(j-1) cell holds more than B
// particles -- when some run of B + 1 consecutive sorted keys around i shares
// j - 1 digits.  So particle i owns the depths L_i < j <= J_i, with
// J_i = min(21, 1 + max over a in [i-B, i] of lcp(key[a], key[a+B])), and its
// node at depth j is internal iff j < J_i.  Likewise (with G for B) the walk
// group of i's chain sits at depth min(J_i, 1 + max lcp over the G-runs).
//
// Nodes are numbered depth by depth, each depth in Morton order, so the
// children of a node are consecutive: a count pass per tile of particles, a
// scan of the per-tile counts of each depth, then a pass in which each owner
// writes its nodes.  A node's first child index is the number of depth-(j+1)
// nodes before its start; the child count is the difference to the next node
// of the same depth.  Node boundaries: down to the PM mesh depth m the cell
// ends come from the CSR table of the depth-m Morton cells; deeper, a binary
// search of the keys inside the parent's range.  The numbering depends only
// on the keys (no atomics), so the tree is deterministic.
//
// Node sums in one pass, without a climb: a node's mass and mass-weighted
// position (uint64, exact) are differences of exclusive prefix sums over the
// sorted particles at its range ends (a leaf sums its <= B particles
// directly), giving the rounded integer COM; the largest member
// multiplicity (node softening) starts at 1 everywhere, and only a leaf
// holding a merged particle (k > 1) raises its ancestors' value with
// atomicMax, stopping where an ancestor already holds at least as much (the
// maximum is order-free, so the tree is deterministic).  Walk groups (node
// with <= G particles whose parent holds more, or a leaf) are listed in Morton
// order.
#include "common.cuh"

namespace dzs {
namespace {

constexpr int kTreeTile = 1024;          // particles per block (one per thread)
constexpr int kHalo = 64;                // largest G (walk_group <= 64)
constexpr int kCols = kMaxLevel + 2;     // node counts per depth 0..21, then walk groups
constexpr unsigned kFull = 0xffffffffu;

// octal digits shared by two keys (21 for equal keys); keys are < 2^63
__device__ __forceinline__ int lcp_digits(uint64_t a, uint64_t b) {
  const uint64_t x = a ^ b;
  return x == 0 ? kMaxLevel : (__clzll((long long)x) - 1) / 3;
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

// per particle: L_i, J_i and the group depth g_i (packed into info[i]); per
// tile: the number of nodes of each depth and of walk groups its particles own
__global__ void __launch_bounds__(kTreeTile) k_tree_count(const int32_t* __restrict__ d_n,
                                                          const uint64_t* __restrict__ key, int B, int G,
                                                          int32_t* __restrict__ info, int32_t* __restrict__ tcount,
                                                          int64_t ntiles) {
  __shared__ uint64_t ks[kTreeTile + 2 * kHalo];  // keys t0 - kHalo .. t0 + kTreeTile + kHalo
  __shared__ int8_t wb[kTreeTile + kHalo], wg[kTreeTile + kHalo];  // runs starting at t0 - kHalo + q
  __shared__ int32_t wcnt[kTreeTile / 32][kCols];
  const int64_t n = *d_n;
  const int64_t t0 = (int64_t)blockIdx.x * kTreeTile;
  for (int q = threadIdx.x; q < kTreeTile + 2 * kHalo; q += kTreeTile) {
    const int64_t a = t0 - kHalo + q;
    ks[q] = (a >= 0 && a < n) ? key[a] : 0ull;
  }
  for (int q = threadIdx.x; q < (kTreeTile / 32) * kCols; q += kTreeTile) (&wcnt[0][0])[q] = 0;
  __syncthreads();
  for (int q = threadIdx.x; q < kTreeTile + kHalo; q += kTreeTile) {
    const int64_t a = t0 - kHalo + q;
    wb[q] = (int8_t)((a >= 0 && a + B < n) ? lcp_digits(ks[q], ks[q + B]) : -1);
    wg[q] = (int8_t)((a >= 0 && a + G < n) ? lcp_digits(ks[q], ks[q + G]) : -1);
  }
  __syncthreads();
  const int64_t i = t0 + threadIdx.x;
  const int q = threadIdx.x + kHalo;
  const bool valid = i < n;
  int L = 0, J = -1, g = -1;
  if (valid) {
    L = i > 0 ? lcp_digits(ks[q - 1], ks[q]) : -1;
    int mb = -1, mg = -1;
    for (int d = 0; d <= B; ++d) mb = max(mb, (int)wb[q - d]);
    for (int d = 0; d <= G; ++d) mg = max(mg, (int)wg[q - d]);
    J = min(kMaxLevel, 1 + mb);
    g = min(J, 1 + mg);
    info[i] = (L + 1) | (J << 8) | (g << 16);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const bool owner = valid && L < J;
  const int jlo = __reduce_min_sync(kFull, owner ? L + 1 : kMaxLevel + 1);
  const int jhi = __reduce_max_sync(kFull, owner ? J : -1);
  for (int j = jlo; j <= jhi; ++j) {
    const unsigned b = __ballot_sync(kFull, owner && L < j && j <= J);
    if (lane == 0) wcnt[w][j] = __popc(b);
  }
  const unsigned bg = __ballot_sync(kFull, valid && L < g);
  if (lane == 0) wcnt[w][kCols - 1] = __popc(bg);
  __syncthreads();
  if (threadIdx.x < kCols) {
    int s = 0;
    for (int ww = 0; ww < kTreeTile / 32; ++ww) s += wcnt[ww][threadIdx.x];
    tcount[(int64_t)threadIdx.x * ntiles + blockIdx.x] = s;
  }
}

// block c: exclusive scan of column c of the tile counts, column total to tot[c]
__global__ void k_tree_scan(int32_t* __restrict__ tcount, int64_t ntiles, int32_t* __restrict__ tot) {
  __shared__ int32_t warp_tot[32];
  __shared__ int32_t carry;
  int32_t* col = tcount + (int64_t)blockIdx.x * ntiles;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t b0 = 0; b0 < ntiles; b0 += blockDim.x) {
    const int64_t b = b0 + threadIdx.x;
    const int32_t v = b < ntiles ? col[b] : 0;
    int32_t inc = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t t = __shfl_up_sync(kFull, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
      const int32_t t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
      int32_t ti = t;
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t u = __shfl_up_sync(kFull, ti, o);
        if (lane >= o) ti += u;
      }
      warp_tot[lane] = ti - t;
    }
    __syncthreads();
    const int32_t ex = inc - v + warp_tot[w] + carry;
    if (b < ntiles) col[b] = ex;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = ex + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) tot[blockIdx.x] = carry;
}

// node counts per depth and the group count; a tree above the node capacity
// is not built (error bit, zero nodes and groups)
__global__ void k_tree_totals(int32_t* __restrict__ lvl, int64_t node_cap, uint64_t* __restrict__ counters,
                              uint32_t* __restrict__ err) {
  if (threadIdx.x != 0) return;
  int64_t total = 0;
  for (int j = 0; j <= kMaxLevel; ++j) total += lvl[j];
  if (total > node_cap) {
    atomicOr(err, kErrNodes);
    for (int j = 0; j < kCols; ++j) lvl[j] = 0;
    total = 0;
  }
  counters[2] = (uint64_t)lvl[kCols - 1];
  counters[3] = (uint64_t)total;
}

// every owner writes its nodes: index = (nodes of shallower depths) + (nodes of
// the same depth starting before it); first-child index to cfirst
__global__ void __launch_bounds__(kTreeTile) k_tree_nodes(
    const int32_t* __restrict__ d_n, int64_t cap, const uint64_t* __restrict__ key, const uint32_t* __restrict__ u,
    const int32_t* __restrict__ info, const int32_t* __restrict__ tcount, int64_t ntiles,
    const int32_t* __restrict__ lvl, const int32_t* __restrict__ cstart, int depth_m, int B, Node* __restrict__ nodes,
    int32_t* __restrict__ cfirst, int32_t* __restrict__ parent,
    int32_t* __restrict__ groups) {
  __shared__ int32_t wcnt[kTreeTile / 32][kCols];
  __shared__ int32_t base[kCols];
  const int64_t n = *d_n;
  const int64_t t0 = (int64_t)blockIdx.x * kTreeTile;
  if (threadIdx.x == 0) {
    int32_t s = 0;
    for (int j = 0; j <= kMaxLevel; ++j) {
      base[j] = s + tcount[(int64_t)j * ntiles + blockIdx.x];
      s += lvl[j];
    }
    base[kCols - 1] = tcount[(int64_t)(kCols - 1) * ntiles + blockIdx.x];
    base[0] = s == 0 ? -1 : base[0];  // no tree (empty or over capacity)
  }
  for (int q = threadIdx.x; q < (kTreeTile / 32) * kCols; q += kTreeTile) (&wcnt[0][0])[q] = 0;
  __syncthreads();
  if (base[0] < 0) return;
  const int64_t i = t0 + threadIdx.x;
  const bool valid = i < n;
  int L = 0, J = -1, g = -1;
  if (valid) {
    const int32_t v = info[i];
    L = (v & 0xff) - 1;
    J = (v >> 8) & 0xff;
    g = (v >> 16) & 0xff;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const bool owner = valid && L < J;
  // depths whose ranks this warp needs: its nodes' depths and one below
  const int jlo = __reduce_min_sync(kFull, owner ? L + 1 : kMaxLevel + 1);
  const int jhi = min(kMaxLevel, __reduce_max_sync(kFull, owner ? J + 1 : -1));
  for (int j = jlo; j <= jhi; ++j) {
    const unsigned b = __ballot_sync(kFull, owner && L < j && j <= J);
    if (lane == 0) wcnt[w][j] = __popc(b);
  }
  const unsigned bg = __ballot_sync(kFull, valid && L < g);
  if (lane == 0) wcnt[w][kCols - 1] = __popc(bg);
  __syncthreads();
  // lane c holds the first index of column c for this warp
  int32_t wbase = 0;
  if (lane < kCols) {
    wbase = base[lane];
    for (int ww = 0; ww < w; ++ww) wbase += wcnt[ww][lane];
  }
  const uint64_t k = valid ? key[i] : 0ull;
  const uint32_t ux = valid ? u[i] : 0u, uy = valid ? u[cap + i] : 0u, uz = valid ? u[2 * cap + i] : 0u;
  int32_t prev = -1;      // index of this particle's node one depth up
  int64_t prev_end = 0;   // its end
  int32_t gnode = -1;
  for (int j = jlo; j <= jhi; ++j) {
    const bool mine = owner && L < j && j <= J;
    const unsigned b = __ballot_sync(kFull, mine);
    const int32_t rank = __shfl_sync(kFull, wbase, j) + __popc(b & lt);
    if (prev >= 0) cfirst[prev] = rank;  // depth-j nodes before this particle
    if (!mine) {
      prev = -1;
      continue;
    }
    const int sh = 3 * (kMaxLevel - j);
    const uint64_t pref = k >> sh;
    int64_t end;
    if (j <= depth_m) {
      end = cstart[(pref + 1) << (3 * (depth_m - j))];
    } else {
      int64_t hi = prev >= 0 ? prev_end : (int64_t)cstart[(k >> (3 * (kMaxLevel - depth_m))) + 1];
      if (j == J && J < kMaxLevel) hi = min(hi, i + B + 1);  // a leaf above depth 21 holds <= B
      end = lb(key, i + 1, hi, (pref + 1) << sh);
    }
    const uint32_t half = 1u << (31 - j);
    const uint32_t mask = j == 0 ? 0u : ~((half << 1) - 1u);
    Node c;
    c.cx = (ux & mask) | half;
    c.cy = (uy & mask) | half;
    c.cz = (uz & mask) | half;
    c.comx = c.comy = c.comz = 0;
    c.mass = 0;
    c.kmax = 1;  // every member has k >= 1; raised by the leaves that hold merged particles
    c.start = (int32_t)i;
    c.count = (int32_t)(end - i);
    c.child = j < J ? 0 : -1;  // internal: linked by k_tree_link
    c.meta = (uint32_t)j;
    nodes[rank] = c;
    if (j == 0) parent[rank] = -1;
    if (j == g) gnode = rank;
    prev = rank;
    prev_end = end;
  }
  if (prev >= 0) cfirst[prev] = 0;  // depth 21: no children
  const int32_t gbase = __shfl_sync(kFull, wbase, kCols - 1);  // all lanes take part
  if (valid && L < g) groups[gbase + __popc(bg & lt)] = gnode;
}

// internal nodes: first child and child count (to the next node of the same
// depth, or to the end of the next depth), parent links of the children
__global__ void k_tree_link(const int32_t* __restrict__ lvl, Node* __restrict__ nodes,
                            const int32_t* __restrict__ cfirst, int32_t* __restrict__ parent) {
  __shared__ int32_t lb_[kMaxLevel + 3];
  if (threadIdx.x == 0) {
    int32_t s = 0;
    for (int j = 0; j <= kMaxLevel; ++j) {
      lb_[j] = s;
      s += lvl[j];
    }
    lb_[kMaxLevel + 1] = s;
    lb_[kMaxLevel + 2] = s;
  }
  __syncthreads();
  const int64_t total = lb_[kMaxLevel + 1];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    if (nodes[t].child < 0) continue;
    const int j = (int)(nodes[t].meta & 0xff);
    const int32_t c0 = cfirst[t];
    const int32_t c1 = (t + 1 < lb_[j + 1]) ? cfirst[t + 1] : lb_[j + 2];
    nodes[t].child = c0;
    nodes[t].meta = (uint32_t)j | ((uint32_t)(c1 - c0) << 8);
    for (int32_t q = c0; q < c1; ++q) parent[q] = (int32_t)t;
  }
}

__device__ __forceinline__ void write_mass_com(Node* __restrict__ nodes, int64_t ni, uint64_t K,
                                               const uint64_t (&S)[3]) {
  nodes[ni].mass = (uint32_t)K;
  if (K > 0) {
    nodes[ni].comx = (uint32_t)((2 * S[0] + K) / (2 * K));
    nodes[ni].comy = (uint32_t)((2 * S[1] + K) / (2 * K));
    nodes[ni].comz = (uint32_t)((2 * S[2] + K) / (2 * K));
  }
}

// every node: leaves sum their particles (four loads in flight at a time) and
// raise their ancestors' largest multiplicity when it exceeds 1; internal
// nodes take prefix-sum differences (pre: exclusive [4][cap + 1])
__global__ void k_tree_sums(const int32_t* __restrict__ lvl, int64_t cap, const uint32_t* __restrict__ u,
                            const uint32_t* __restrict__ k, const uint64_t* __restrict__ pre,
                            Node* __restrict__ nodes, const int32_t* __restrict__ parent) {
  int64_t total = 0;
  for (int j = 0; j <= kMaxLevel; ++j) total += lvl[j];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s0 = nodes[t].start, cnt = nodes[t].count, child = nodes[t].child;
    uint64_t K = 0, S[3] = {0, 0, 0};
    if (child >= 0) {
      const int64_t e = (int64_t)s0 + cnt;
      K = pre[e] - pre[s0];
      for (int ax = 0; ax < 3; ++ax) S[ax] = pre[(int64_t)(1 + ax) * (cap + 1) + e] - pre[(int64_t)(1 + ax) * (cap + 1) + s0];
      write_mass_com(nodes, t, K, S);
      continue;
    }
    uint32_t kmax = 0;
    const int64_t i1 = (int64_t)s0 + cnt;
    for (int64_t i0 = s0; i0 < i1; i0 += 4) {
      uint32_t kk[4], ux[4], uy[4], uz[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const bool in = i0 + q < i1;
        const int64_t i = in ? i0 + q : i0;
        kk[q] = in ? k[i] : 0u;
        ux[q] = u[i];
        uy[q] = u[cap + i];
        uz[q] = u[2 * cap + i];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        K += kk[q];
        kmax = max(kmax, kk[q]);
        S[0] += (uint64_t)kk[q] * ux[q];
        S[1] += (uint64_t)kk[q] * uy[q];
        S[2] += (uint64_t)kk[q] * uz[q];
      }
    }
    write_mass_com(nodes, t, K, S);
    nodes[t].kmax = kmax;
    if (kmax > 1)
      for (int32_t a = parent[t]; a >= 0; a = parent[a])
        if (atomicMax(&nodes[a].kmax, kmax) >= kmax) break;  // the rest is raised already (or being raised)
  }
}

}  // namespace

void launch_tree(dzs_ctx* c) {
  c->launches += 6;
  Buffers& B = c->B;
  // the depth-m Morton cell table (also the PM deposit's)
  launch_cell_start(c);
  const int64_t ntiles = (c->cap + kTreeTile - 1) / kTreeTile;
  int32_t* info = B.group_head;       // [cap] per-particle L, J, g
  int32_t* tcount = B.iscan;          // [kCols][ntiles] tile counts, then offsets
  int32_t* cfirst = B.cfirst;         // [node_cap]
  k_tree_count<<<(unsigned)ntiles, kTreeTile, 0, c->stream>>>(B.n, B.key, c->P.leaf_bucket, c->P.walk_group, info,
                                                              tcount, ntiles);
  k_tree_scan<<<kCols, 1024, 0, c->stream>>>(tcount, ntiles, B.lvl_count);
  k_tree_totals<<<1, 32, 0, c->stream>>>(B.lvl_count, c->node_cap, B.counters, B.err);
  k_tree_nodes<<<(unsigned)ntiles, kTreeTile, 0, c->stream>>>(B.n, c->cap, B.key, B.u, info, tcount, ntiles,
                                                              B.lvl_count, B.cell_start, c->logM, c->P.leaf_bucket,
                                                              B.nodes, cfirst, B.parent, B.groups);
  k_tree_link<<<grid_for(c->node_cap, kThreads, 8), kThreads, 0, c->stream>>>(B.lvl_count, B.nodes, cfirst,
                                                                                     B.parent);
  launch_mass_prefix(c);
  k_tree_sums<<<grid_for(c->node_cap, kThreads, 8), kThreads, 0, c->stream>>>(B.lvl_count, c->cap, B.u, B.k,
                                                                               B.prefix, B.nodes, B.parent);
}

}  // namespace dzs
