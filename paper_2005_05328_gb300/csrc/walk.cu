// walk.cu -- short-range tree force (paper Sec. 2.1: monopole-only oct-tree
// joined to the PM force by the Gaussian split; Eq. 1: a node is opened when
// l_n / d >= theta; Sec. 2.2: softening rescaled by (M / M_init)^(1/3)),
// fused with the closing kick.
//
// One warp per walk group (a node with <= G particles whose parent holds more,
// or a leaf); lane l owns particle start + l.  The warp walks the tree against
// the group's cube with a shared-memory stack, up to 32 nodes per round (one
// per lane):
//   skip   the node's cube is farther than r_cut from the group cube;
//   open   the cubes touch, or l_n >= theta d(COM_n, group cube);
//   accept otherwise: the monopole (COM, mass, softening) joins the list.
// Opened leaves put their particles on the list.  Cube gaps and COM distances
// are exact integers; the two comparisons use FP64 as the CPU reference does,
// so both sides build the same interaction set.  The list lives in shared
// memory and is evaluated by all lanes (each for its own particle) whenever it
// fills: softened pair force times T(r) = erfc(r / 2 r_s) + r / (r_s sqrt(pi))
// exp(-r^2 / 4 r_s^2), zero at r = 0 or r >= r_cut.
#include <cmath>

#include "common.cuh"

namespace dzs {
namespace {

constexpr int kWarps = 4;
constexpr int kStack = 1024;
constexpr int kList = 512;

template <class R>
struct WalkSmem {
  int32_t stack[kWarps][kStack];
  uint32_t lx[kWarps][kList], ly[kWarps][kList], lz[kWarps][kList];
  R lm[kWarps][kList];  // G m of the entry
  R lh[kWarps][kList];  // spline radius 2.8 eps of the entry
};

template <class R>
struct WalkConst {
  R scale;       // L / 2^32
  R rcut2;       // r_cut^2
  R inv2rs;      // 1 / (2 r_s)
  R c1;          // 1 / (r_s sqrt(pi))
  R gm0;         // G m0
  R h0;          // 2.8 eps0
  double rcut_lat2;
  double theta;
  R kick;        // closing kick factor (0: none)
  int B;
  int close;
  int tree;
};

template <class R>
__device__ __forceinline__ R spline_fac(R r, R h) {
  // cubic-spline softened 1 / r^3 (enclosed kernel mass / r^3)
  R q = r / h, h3 = h * h * h;
  if (q < (R)0.5) return ((R)(32.0 / 3.0) + q * q * ((R)32.0 * q - (R)38.4)) / h3;
  return ((R)(64.0 / 3.0) - (R)48.0 * q + (R)38.4 * q * q - (R)(32.0 / 3.0) * q * q * q -
          (R)(1.0 / 15.0) / (q * q * q)) / h3;
}

__device__ __forceinline__ float erfc_r(float x) { return erfcf(x); }
__device__ __forceinline__ double erfc_r(double x) { return erfc(x); }
__device__ __forceinline__ float exp_r(float x) { return __expf(x); }
__device__ __forceinline__ double exp_r(double x) { return exp(x); }

template <class R>
__device__ __forceinline__ void eval_list(const WalkSmem<R>& sm, int w, int len, bool active, uint32_t xi,
                                          uint32_t yi, uint32_t zi, R hi, const WalkConst<R>& C, R& ax,
                                          R& ay, R& az) {
  if (!active) return;
  for (int e = 0; e < len; ++e) {
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
      R x = r * C.inv2rs;
      R t = erfc_r(x) + r * C.c1 * exp_r(-x * x);
      R f = sm.lm[w][e] * fac * t;
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
      const int64_t i = (int64_t)gn.start + c0 + lane;
      const bool active = c0 + lane < gn.count;
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
            const int64_t ln = 1ll << (32 - (int)(nd.meta & 0xff));
            bool touch = true;
            uint64_t dist2 = 0, dcom2 = 0;
            const uint32_t cn[3] = {nd.cx, nd.cy, nd.cz}, cg[3] = {gn.cx, gn.cy, gn.cz};
            const uint32_t cm[3] = {nd.comx, nd.comy, nd.comz};
#pragma unroll
            for (int ax3 = 0; ax3 < 3; ++ax3) {
              int64_t dc = (int32_t)(cn[ax3] - cg[ax3]);
              dc = dc < 0 ? -dc : dc;
              int64_t gap = dc - (lg + ln) / 2;
              if (gap > 0) {
                touch = false;
                dist2 += (uint64_t)gap * (uint64_t)gap;
              }
              int64_t dm = (int32_t)(cm[ax3] - cg[ax3]);
              dm = (dm < 0 ? -dm : dm) - lg / 2;
              if (dm > 0) dcom2 += (uint64_t)dm * (uint64_t)dm;
            }
            if (touch || (double)dist2 <= C.rcut_lat2) {
              bool open = touch || ((double)ln >= C.theta * sqrt((double)dcom2));
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
          int cnt = (leaf && nd.count <= C.B) ? nd.count : 0;
          int exl = cnt;
          for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, exl, o);
            if (lane >= o) exl += t;
          }
          int totl = __shfl_sync(0xffffffffu, exl, 31);
          exl -= cnt;
          for (int q = 0; q < cnt; ++q) {
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
                eval_list(sm, w, len, active, xi, yi, zi, hi, C, ax, ay, az);
                npairs += active ? (unsigned long long)len : 0ull;
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
            eval_list(sm, w, len, active, xi, yi, zi, hi, C, ax, ay, az);
            npairs += active ? (unsigned long long)len : 0ull;
            len = 0;
            __syncwarp();
          }
        }
        __syncwarp();
        eval_list(sm, w, len, active, xi, yi, zi, hi, C, ax, ay, az);
        npairs += active ? (unsigned long long)len : 0ull;
        __syncwarp();
      }
      if (active) {
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
  C.c1 = (R)(1.0 / (c->rs * std::sqrt(M_PI)));
  C.gm0 = (R)c->gm0;
  C.h0 = (R)(2.8 * c->eps0);
  C.rcut_lat2 = c->rcut_lat2;
  C.theta = c->P.theta;
  C.kick = close_kick ? (R)c->T.kick2[step] : (R)0;
  C.B = c->P.leaf_bucket;
  C.close = close_kick ? 1 : 0;
  C.tree = tree ? 1 : 0;
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
