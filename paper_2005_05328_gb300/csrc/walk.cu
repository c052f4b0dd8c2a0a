// walk.cu -- short-range tree force (paper Sec. 2.1: monopole-only oct-tree
// joined to the PM force by the Gaussian split; Eq. 1: a node is opened when
// l_n / d >= theta; Sec. 2.2: softening rescaled by (M / M_init)^(1/3)),
// fused with the closing kick.
//
// One warp per walk group (a node with <= G particles whose parent holds more,
// or a leaf).  The warp walks the tree against the group's cube with a
// shared-memory stack, up to 32 nodes per round (one per lane):
//   skip   the node's cube is farther than r_cut from the group cube;
//   open   the cubes touch, or l_n >= theta d(COM_n, group cube);
//   accept otherwise: the monopole (COM, mass, softening) joins the list.
// Opened leaves put their particles on the list.  Cube gaps and COM distances
// are exact integers.  The FP64 comparisons that define skip and open
// ((double)gap^2 <= r_cut^2, (double)l >= theta sqrt((double)d^2)) are
// monotone in the integer d^2, so the host turns each into an exact integer
// threshold once per context: the walk compares integers only and builds the
// same interaction set as the CPU reference, with no FP64 in the walk.
// The list lives in shared memory; when it fills, all 32 lanes evaluate it:
// a group of c particles gets 32 / next_pow2(c) lanes per particle, each lane
// summing every S-th entry, combined by a fixed xor-shuffle tree (the result
// is deterministic).  Pair force: softened 1/r^3 times
// T(r) = erfc(x) + (2/sqrt(pi)) x exp(-x^2), x = r / 2 r_s, zero at r = 0 and
// r >= r_cut.  FP32 evaluates T = exp(-x^2) Q(x) with a fitted polynomial
// (gen_split_poly.py, relative error 3.3e-7); FP64 calls erfc and exp.
#include <cmath>

#include "common.cuh"

namespace dzs {
namespace {

constexpr int kWarps = 4;
constexpr int kStack = 1024;
constexpr int kList = 512;

// Q(t) power-series coefficients, t = 2 x / 2.5 - 1; FP32 rel. error 3.32e-07
// (generated by gen_split_poly.py)
__constant__ float kSplitPoly[12] = {1.778296833e+00f, 1.149446721e+00f, 1.668713091e-01f, -9.808575506e-02f,
                                     5.369898964e-02f, -2.768828264e-02f, 1.372957384e-02f, -6.415871732e-03f,
                                     2.482135905e-03f, -1.056264300e-03f, 7.980994871e-04f, -3.233674216e-04f};
constexpr float kSplitXMax = 2.5f;

template <class R>
struct WalkSmem {
  int32_t stack[kWarps][kStack];
  uint32_t lx[kWarps][kList], ly[kWarps][kList], lz[kWarps][kList];
  R lm[kWarps][kList];  // G m of the entry
  R lh[kWarps][kList];  // spline radius 2.8 eps of the entry
};

template <class R>
struct WalkConst {
  R scale;  // L / 2^32
  R rcut2;  // r_cut^2
  R inv2rs;  // 1 / (2 r_s)
  R c1;      // 2 / sqrt(pi)
  R gm0;     // G m0
  R h0;      // 2.8 eps0
  R kick;    // closing kick factor
  uint64_t skip_d2;                   // not skipped iff cube gap^2 <= skip_d2
  uint64_t open_d2[kMaxLevel + 1];    // opened iff COM distance^2 <= open_d2[level]
  int B;
  int close;
  int tree;
  int poly;  // FP32: use the fitted split polynomial (x_max <= 2.5)
};

template <class R>
__device__ __forceinline__ R spline_fac(R r, R h) {
  // cubic-spline softened 1 / r^3 (enclosed kernel mass / r^3)
  R q = r / h, h3 = h * h * h;
  if (q < (R)0.5) return ((R)(32.0 / 3.0) + q * q * ((R)32.0 * q - (R)38.4)) / h3;
  return ((R)(64.0 / 3.0) - (R)48.0 * q + (R)38.4 * q * q - (R)(32.0 / 3.0) * q * q * q -
          (R)(1.0 / 15.0) / (q * q * q)) / h3;
}

__device__ __forceinline__ float split_factor(float x, int poly) {
  if (poly) {
    float t = x * (2.0f / kSplitXMax) - 1.0f;
    float q = kSplitPoly[11];
#pragma unroll
    for (int i = 10; i >= 0; --i) q = fmaf(q, t, kSplitPoly[i]);
    return __expf(-x * x) * q;
  }
  return erfcf(x) + 1.1283791670955126f * x * __expf(-x * x);
}

__device__ __forceinline__ double split_factor(double x, int) {
  return erfc(x) + 1.1283791670955126 * x * exp(-x * x);
}

template <class R>
__device__ __forceinline__ void eval_list(const WalkSmem<R>& sm, int w, int len, int sub, int S, bool active,
                                          uint32_t xi, uint32_t yi, uint32_t zi, R hi, const WalkConst<R>& C,
                                          R& ax, R& ay, R& az) {
  if (!active) return;
  for (int e = sub; e < len; e += S) {
    R dx = (R)(int32_t)(sm.lx[w][e] - xi) * C.scale;
    R dy = (R)(int32_t)(sm.ly[w][e] - yi) * C.scale;
    R dz = (R)(int32_t)(sm.lz[w][e] - zi) * C.scale;
    R r2 = dx * dx + dy * dy + dz * dz;
    if (r2 > (R)0 && r2 < C.rcut2) {
      R r = sqrt(r2);
      R h = sm.lh[w][e] > hi ? sm.lh[w][e] : hi;
      R fac;
      if (r >= h) {
        R ir = (R)1 / r;
        fac = ir * ir * ir;
      } else {
        fac = spline_fac(r, h);
      }
      R f = sm.lm[w][e] * fac * split_factor(r * C.inv2rs, C.poly);
      ax += f * dx;
      ay += f * dy;
      az += f * dz;
    }
  }
}

template <class R>
__global__ void __launch_bounds__(kWarps * 32) k_walk(
    const int32_t* __restrict__ groups, const uint64_t* __restrict__ counters, unsigned int* __restrict__ next,
    const Node* __restrict__ nodes, int64_t cap, const uint32_t* __restrict__ u, const uint32_t* __restrict__ k,
    R* __restrict__ p, R* __restrict__ g, WalkConst<R> C, uint32_t* __restrict__ err,
    unsigned long long* __restrict__ pairs) {
  extern __shared__ unsigned char smem_raw[];
  WalkSmem<R>& sm = *reinterpret_cast<WalkSmem<R>*>(smem_raw);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t ngroups = (int64_t)counters[2];
  unsigned long long npairs = 0;
  const int flush_at = kList - 32 * (C.B > 1 ? C.B : 1) - 32;
  for (;;) {
    int64_t gi = 0;
    if (lane == 0) gi = atomicAdd(next, 1u);
    gi = __shfl_sync(0xffffffffu, gi, 0);
    if (gi >= ngroups) break;
    const Node gn = nodes[groups[gi]];
    const int glevel = gn.meta & 0xff;
    const int64_t lg = 1ll << (32 - glevel);
    for (int c0 = 0; c0 < gn.count; c0 += 32) {
      // lanes per particle S = 32 / next_pow2(particles in this chunk)
      const int cnt = gn.count - c0 < 32 ? gn.count - c0 : 32;
      const int S = 32 >> (32 - __clz(cnt - 1 > 0 ? cnt - 1 : 0));
      const int mine = lane / S, sub = lane % S;
      const int64_t i = (int64_t)gn.start + c0 + mine;
      const bool active = mine < cnt;
      uint32_t xi = 0, yi = 0, zi = 0;
      R hi = 0;
      if (active) {
        xi = u[i];
        yi = u[cap + i];
        zi = u[2 * cap + i];
        hi = C.h0 * cbrt((R)k[i]);
      }
      R ax = 0, ay = 0, az = 0;
      if (C.tree) {
        int top = 0, len = 0;
        if (lane == 0) sm.stack[w][0] = 0;
        top = 1;
        __syncwarp();
        while (top > 0) {
          const int npop = top < 32 ? top : 32;
          int ni = lane < npop ? sm.stack[w][top - npop + lane] : -1;
          top -= npop;
          __syncwarp();
          bool acc = false, leaf = false, inner = false;
          Node nd;
          if (ni >= 0) {
            nd = nodes[ni];
            const int nlevel = (int)(nd.meta & 0xff);
            const int64_t ln = 1ll << (32 - nlevel);
            bool touch = true;
            uint64_t dist2 = 0, dcom2 = 0;
            const uint32_t cn[3] = {nd.cx, nd.cy, nd.cz}, cg[3] = {gn.cx, gn.cy, gn.cz};
            const uint32_t cm[3] = {nd.comx, nd.comy, nd.comz};
#pragma unroll
            for (int a3 = 0; a3 < 3; ++a3) {
              int64_t dc = (int32_t)(cn[a3] - cg[a3]);
              dc = dc < 0 ? -dc : dc;
              int64_t gap = dc - (lg + ln) / 2;
              if (gap > 0) {
                touch = false;
                dist2 += (uint64_t)gap * (uint64_t)gap;
              }
              int64_t dm = (int32_t)(cm[a3] - cg[a3]);
              dm = (dm < 0 ? -dm : dm) - lg / 2;
              if (dm > 0) dcom2 += (uint64_t)dm * (uint64_t)dm;
            }
            if (touch || dist2 <= C.skip_d2) {
              bool open = touch || dcom2 <= C.open_d2[nlevel];
              if (!open)
                acc = true;
              else if (nd.child < 0)
                leaf = true;
              else
                inner = true;
            }
          }
          // accepted monopoles
          unsigned am = __ballot_sync(0xffffffffu, acc);
          if (acc) {
            int pos = len + __popc(am & lt);
            sm.lx[w][pos] = nd.comx;
            sm.ly[w][pos] = nd.comy;
            sm.lz[w][pos] = nd.comz;
            sm.lm[w][pos] = C.gm0 * (R)nd.mass;
            sm.lh[w][pos] = C.h0 * cbrt((R)nd.kmax);
          }
          len += __popc(am);
          // children of opened inner nodes onto the stack
          int nch = inner ? (int)((nd.meta >> 8) & 0xff) : 0;
          int ex = nch;
          for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, ex, o);
            if (lane >= o) ex += t;
          }
          int tot = __shfl_sync(0xffffffffu, ex, 31);
          ex -= nch;
          if (top + tot > kStack) {
            if (lane == 0) atomicOr(err, kErrStack);
            nch = 0;
            tot = 0;
          }
          for (int q = 0; q < nch; ++q) sm.stack[w][top + ex + q] = nd.child + q;
          top += tot;
          // particles of opened small leaves
          int lc = (leaf && nd.count <= C.B) ? nd.count : 0;
          int exl = lc;
          for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, exl, o);
            if (lane >= o) exl += t;
          }
          int totl = __shfl_sync(0xffffffffu, exl, 31);
          exl -= lc;
          for (int q = 0; q < lc; ++q) {
            int pos = len + exl + q;
            int64_t j = (int64_t)nd.start + q;
            sm.lx[w][pos] = u[j];
            sm.ly[w][pos] = u[cap + j];
            sm.lz[w][pos] = u[2 * cap + j];
            uint32_t kj = k[j];
            sm.lm[w][pos] = C.gm0 * (R)kj;
            sm.lh[w][pos] = C.h0 * cbrt((R)kj);
          }
          len += totl;
          __syncwarp();
          // big leaves (depth 21, more than B particles): stream through
          unsigned bm = __ballot_sync(0xffffffffu, leaf && nd.count > C.B);
          while (bm) {
            int src = __ffs(bm) - 1;
            bm &= bm - 1;
            int bs = __shfl_sync(0xffffffffu, nd.start, src);
            int bc = __shfl_sync(0xffffffffu, nd.count, src);
            for (int q0 = 0; q0 < bc; q0 += 32) {
              if (len + 32 > kList) {
                __syncwarp();
                eval_list(sm, w, len, sub, S, active, xi, yi, zi, hi, C, ax, ay, az);
                npairs += (active && sub == 0) ? (unsigned long long)len : 0ull;
                len = 0;
                __syncwarp();
              }
              int m = bc - q0 < 32 ? bc - q0 : 32;
              if (lane < m) {
                int64_t j = (int64_t)bs + q0 + lane;
                sm.lx[w][len + lane] = u[j];
                sm.ly[w][len + lane] = u[cap + j];
                sm.lz[w][len + lane] = u[2 * cap + j];
                uint32_t kj = k[j];
                sm.lm[w][len + lane] = C.gm0 * (R)kj;
                sm.lh[w][len + lane] = C.h0 * cbrt((R)kj);
              }
              len += m;
              __syncwarp();
            }
          }
          if (len > flush_at) {
            eval_list(sm, w, len, sub, S, active, xi, yi, zi, hi, C, ax, ay, az);
            npairs += (active && sub == 0) ? (unsigned long long)len : 0ull;
            len = 0;
            __syncwarp();
          }
        }
        __syncwarp();
        eval_list(sm, w, len, sub, S, active, xi, yi, zi, hi, C, ax, ay, az);
        npairs += (active && sub == 0) ? (unsigned long long)len : 0ull;
        __syncwarp();
        // combine the S partial sums of each particle (fixed xor tree)
        for (int o = 1; o < S; o <<= 1) {
          ax += __shfl_xor_sync(0xffffffffu, ax, o);
          ay += __shfl_xor_sync(0xffffffffu, ay, o);
          az += __shfl_xor_sync(0xffffffffu, az, o);
        }
      }
      if (active && sub == 0) {
        R gx = g[i] + ax, gy = g[cap + i] + ay, gz = g[2 * cap + i] + az;
        g[i] = gx;
        g[cap + i] = gy;
        g[2 * cap + i] = gz;
        if (C.close) {
          p[i] += gx * C.kick;
          p[cap + i] += gy * C.kick;
          p[2 * cap + i] += gz * C.kick;
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) npairs += __shfl_down_sync(0xffffffffu, npairs, o);
  if (lane == 0 && npairs) atomicAdd(pairs, npairs);
}

template <class R>
void walk_impl(dzs_ctx* c, bool tree, bool close_kick, int step) {
  WalkConst<R> C;
  C.scale = (R)c->scale;
  C.rcut2 = (R)(c->rcut * c->rcut);
  C.inv2rs = (R)(1.0 / (2.0 * c->rs));
  C.c1 = (R)(2.0 / std::sqrt(M_PI));
  C.gm0 = (R)c->gm0;
  C.h0 = (R)(2.8 * c->eps0);
  C.kick = close_kick ? (R)c->T.kick2[step] : (R)0;
  C.skip_d2 = c->walk_skip_d2;
  for (int l = 0; l <= kMaxLevel; ++l) C.open_d2[l] = c->walk_open_d2[l];
  C.B = c->P.leaf_bucket;
  C.close = close_kick ? 1 : 0;
  C.tree = tree ? 1 : 0;
  C.poly = (c->P.rcut_rs / 2.0 <= (double)kSplitXMax) ? 1 : 0;
  size_t sm = sizeof(WalkSmem<R>);
  static bool attr_done[2] = {false, false};
  if (!attr_done[sizeof(R) == 8]) {
    cudaFuncSetAttribute(k_walk<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr_done[sizeof(R) == 8] = true;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk<R>, kWarps * 32, sm);
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->dev);
  int grid = (per_sm > 0 ? per_sm : 1) * (nsm > 0 ? nsm : 1);
  unsigned int* next = (unsigned int*)(c->B.counters + 6);
  cudaMemsetAsync(next, 0, sizeof(unsigned int), c->stream);
  k_walk<R><<<grid, kWarps * 32, sm, c->stream>>>(c->B.groups, c->B.counters, next, c->B.nodes, c->cap, c->B.u,
                                                  c->B.k, (R*)c->B.p, (R*)c->B.g, C, c->B.err,
                                                  (unsigned long long*)(c->B.counters + 4));
}

}  // namespace

void launch_walk(dzs_ctx* c, bool tree, bool close_kick, int step) {
  c->launches += 1;
  if (c->fp64)
    walk_impl<double>(c, tree, close_kick, step);
  else
    walk_impl<float>(c, tree, close_kick, step);
}

}  // namespace dzs
