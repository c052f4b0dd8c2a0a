// walk.cu -- short-range tree force (paper Sec. 2.1: monopole-only oct-tree
// joined to the PM force by the Gaussian split; Eq. 1: a node is opened when
// l_n / d >= theta; Sec. 2.2: softening rescaled by (M / M_init)^(1/3)),
// fused with the closing kick.
//
// One warp per walk group (a node with <= G particles whose parent holds more,
// or a leaf).  The warp walks the tree against the group's cube with a
// shared-memory stack, up to 32 nodes per round (one per lane), starting from
// the frontier depth f: the deepest depth above which no node can be accepted
// (a node of side l whose cube is within r_cut of the group cube has its COM
// within r_cut + sqrt(3) l, which opens it while that is <= l / theta), and
// whose cells are at least r_cut wide.  From the root the walk would only open
// or skip nodes above f, so it starts instead from the depth-f nodes of the 27
// cells around the group's depth-f cell (or the shallower leaves covering
// them, each once): the same nodes are tested and the same interaction set is
// built, without the first rounds of the descent.  Groups above depth f start
// at the root.  Deeper still, a group at depth >= F - 1 (F = f + 2, else
// f + 1: at most 6 depth-F cells per axis) starts from the depth-F nodes of
// the cells within r_cut of its cube along every axis, when each of their
// ancestors between f and F is "always opened" (its COM is close enough to
// its cube centre that every group cube within r_cut of the node opens it):
// the walk from f would open or skip those ancestors, so again the same nodes
// are tested; otherwise the group falls back to the depth-f cells.  Per node:
//   skip   the node's cube is farther than r_cut from the group cube;
//   open   the cubes touch, or l_n >= theta d(COM_n, group cube);
//   accept otherwise: the monopole (COM, mass, softening) joins the list,
//          unless its COM lies farther than r_cut from the group cube.
// Opened leaves put their particles on the list, except those farther than
// r_cut from the group cube (such a monopole or particle acts on no particle
// of the group).  Cube gaps and COM distances are exact integers.  The FP64
// comparisons that define skip and open ((double)gap^2 <= r_cut^2,
// (double)l >= theta sqrt((double)d^2)) are monotone in the integer d^2, so
// the host turns each into an exact integer threshold once per context: the
// walk compares integers only (FP32 sums decide unless within 2^-20 of a
// threshold, where the uint64 sum decides) and builds the same interaction
// set as the CPU reference, with no FP64 in the traversal.
// The list lives in shared memory and is evaluated between rounds, when it
// holds more than 172 entries (a round adds at most 32 monopoles and the
// leaves that fit; leaves that do not fit wait on the stack).  A group of c
// particles puts every lane to work: lane -> particle m = lane mod c, the
// S_m lanes of particle m each taking every S_m-th entry.  Entries are taken
// 32 at a time: a cheap pass tests r < r_cut into a bit mask, then only the
// pairs in range get the force arithmetic (the warp iterates as often as its
// busiest lane has pairs in range); the lanes of a particle are combined by a
// fixed shuffle tree (the result is deterministic).  Pair force: softened
// 1/r^3 times T(r) = erfc(x) + (2/sqrt(pi)) x exp(-x^2), x = r / 2 r_s, zero
// at r = 0 and r >= r_cut.  FP32 evaluates T = exp(-x^2) Q(x) with a fitted
// polynomial (gen_split_poly.py, relative error 3.3e-7); FP64 calls erfc and
// exp.
#include <cmath>

#include "common.cuh"

namespace dzs {
namespace {

// shared memory sets the occupancy (8 blocks of 4 warps per SM in FP32, 64
// registers): stack 512 entries (deepest use measured 329; an overflow sets an
// error bit), list 236 entries (8 blocks measured 2% faster than 7 blocks
// with 300-entry lists)
constexpr int kWarps = 4;
constexpr int kStack = 512;
constexpr int kList = 236;

// Q(t) power-series coefficients, t = 2 x / 2.5 - 1; FP32 rel. error 3.32e-07
// (generated by gen_split_poly.py)
__constant__ float kSplitPoly[12] = {1.778296833e+00f, 1.149446721e+00f, 1.668713091e-01f, -9.808575506e-02f,
                                     5.369898964e-02f, -2.768828264e-02f, 1.372957384e-02f, -6.415871732e-03f,
                                     2.482135905e-03f, -1.056264300e-03f, 7.980994871e-04f, -3.233674216e-04f};
constexpr float kSplitXMax = 2.5f;

// interaction-list entry: lattice position and G m / s^2 (lattice units)
template <class R>
struct Entry;
template <>
struct __align__(16) Entry<float> {
  uint32_t x, y, z;
  float m;
};
template <>
struct __align__(8) Entry<double> {
  uint32_t x, y, z, pad;
  double m;
};

// list entry in shared memory: FP32 holds the offset from the group cube's
// centre in lattice units, converted once when the entry is listed (a pair
// test is then three FP32 subtractions; every listed entry lies within r_cut
// of the cube, so the offset keeps its lattice precision to a few units);
// FP64 holds the exact lattice position (pair offsets are exact integers)
template <class R>
struct LEntry;
template <>
struct __align__(16) LEntry<float> {
  float x, y, z, m;
};
template <>
struct __align__(8) LEntry<double> {
  uint32_t x, y, z, pad;
  double m;
};

// the lane's particle in the same representation
template <class R>
struct Pos;
template <>
struct Pos<float> {
  float x, y, z;
};
template <>
struct Pos<double> {
  uint32_t x, y, z;
};

__device__ __forceinline__ LEntry<float> make_entry(uint32_t ux, uint32_t uy, uint32_t uz, float m,
                                                    const uint32_t (&cg)[3]) {
  LEntry<float> E;
  E.x = (float)(int32_t)(ux - cg[0]);
  E.y = (float)(int32_t)(uy - cg[1]);
  E.z = (float)(int32_t)(uz - cg[2]);
  E.m = m;
  return E;
}
__device__ __forceinline__ LEntry<double> make_entry(uint32_t ux, uint32_t uy, uint32_t uz, double m,
                                                     const uint32_t (&)[3]) {
  LEntry<double> E;
  E.x = ux;
  E.y = uy;
  E.z = uz;
  E.pad = 0;
  E.m = m;
  return E;
}
template <class R>
__device__ __forceinline__ Pos<R> make_pos(uint32_t x, uint32_t y, uint32_t z, const uint32_t (&cg)[3]);
template <>
__device__ __forceinline__ Pos<float> make_pos<float>(uint32_t x, uint32_t y, uint32_t z, const uint32_t (&cg)[3]) {
  return Pos<float>{(float)(int32_t)(x - cg[0]), (float)(int32_t)(y - cg[1]), (float)(int32_t)(z - cg[2])};
}
template <>
__device__ __forceinline__ Pos<double> make_pos<double>(uint32_t x, uint32_t y, uint32_t z, const uint32_t (&)[3]) {
  return Pos<double>{x, y, z};
}

template <class R>
struct WalkSmem {
  int32_t stack[kWarps][kStack];
  LEntry<R> e[kWarps][kList];
  R h[kWarps][kList];  // spline radius 2.8 eps of the entry (lattice units)
};

// everything in lattice units (s = L / 2^32): a = sum (G m / s^2) X fac(R) T(s R)
template <class R>
struct WalkConst {
  R rcut2;   // (r_cut / s)^2
  R inv2rs;  // s / (2 r_s)
  R tcoef;   // (s / 2 r_s) * 2 / x_max (polynomial variable t = r tcoef - 1)
  R nl2;     // -log2(e) (s / 2 r_s)^2
  R gm0;     // G m0 / s^2
  R kick;    // closing kick factor
  uint64_t skip_d2;                 // not skipped iff cube gap^2 <= skip_d2
  uint64_t open_d2[kMaxLevel + 1];  // opened iff COM distance^2 <= open_d2[level]
  float skip_lo, skip_hi;           // FP32 bounds of skip_d2 (relative margin 2^-20)
  float open_lo[kMaxLevel + 1], open_hi[kMaxLevel + 1];
  int B;
  int close;
  int tree;
  int poly;  // FP32: use the fitted split polynomial (x_max <= 2.5)
  int front;                  // frontier depth f (0: start at the root)
  const int32_t* ftab;        // [2^f]^3 row-major: node of each depth-f cell, -1 if empty
  int frontF;                 // window frontier depth F > f (0: none)
  uint32_t rcx;               // largest integer gap with gap^2 <= skip_d2
  const int32_t* ftabF;       // [2^F]^3: node of each depth-F cell (or the leaf above it), -1 if empty
  const unsigned long long* hmax;  // bits of the largest spline radius of any merged particle or node (device)
  R h0;                            // spline radius of multiplicity 1
  const uint8_t* fspanF;      // its F - depth, bit 7: an ancestor at depths [f, F) may accept
};

__device__ __forceinline__ uint64_t exact_d2(const uint32_t (&v)[3]) {
  return (uint64_t)v[0] * v[0] + (uint64_t)v[1] * v[1] + (uint64_t)v[2] * v[2];
}

// FP32: no division (1/h by the hardware reciprocal approximation, 1/q = h / r
// from the rsqrt the pair already has) and no slow path, so that the rarely
// taken branch adds little to the pair loop
__device__ __forceinline__ float rcp_approx(float v) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v));
  return y;
}
__device__ __forceinline__ float spline_fac_ir(float r, float ir, float h) {
  const float ih = rcp_approx(h), q = r * ih, ih3 = ih * ih * ih;
  if (q < 0.5f) return fmaf(q * q, fmaf(32.0f, q, -38.4f), 32.0f / 3.0f) * ih3;
  const float iq = h * ir, iq3 = iq * iq * iq;
  const float poly = fmaf(q, fmaf(q, fmaf(q, -32.0f / 3.0f, 38.4f), -48.0f), 64.0f / 3.0f);
  return fmaf(-1.0f / 15.0f, iq3, poly) * ih3;
}

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

// exp(-x^2) = 2^(r^2 * nl2) with nl2 = -log2(e) (s / 2 r_s)^2: one multiply from r^2
__device__ __forceinline__ float ex2_approx(float v) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v));
  return y;
}

__device__ __forceinline__ double split_factor(double x, int) {
  return erfc(x) + 1.1283791670955126 * x * exp(-x * x);
}

// r^2 >= 1 lattice unit^2 here (no denormals): the plain hardware rsqrt
__device__ __forceinline__ void inv_and_r(float r2, float& r, float& ir) {
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(ir) : "f"(r2));
  r = r2 * ir;
}
__device__ __forceinline__ void inv_and_r(double r2, double& r, double& ir) {
  r = sqrt(r2);
  ir = 1.0 / r;
}

// squared lattice distance of entry E from the lane's particle P: FP32 from
// the two offsets from the group centre, FP64 from the exact int32
// minimum-image offsets
__device__ __forceinline__ float entry_r2(const LEntry<float>& E, const Pos<float>& P, float& dx, float& dy,
                                          float& dz) {
  dx = E.x - P.x;
  dy = E.y - P.y;
  dz = E.z - P.z;
  return dx * dx + dy * dy + dz * dz;
}
__device__ __forceinline__ double entry_r2(const LEntry<double>& E, const Pos<double>& P, double& dx, double& dy,
                                           double& dz) {
  dx = (double)(int32_t)(E.x - P.x);
  dy = (double)(int32_t)(E.y - P.y);
  dz = (double)(int32_t)(E.z - P.z);
  return dx * dx + dy * dy + dz * dz;
}

// 0 < r2 < r_cut^2 (the self pair has r2 = 0): on the FP32 bit patterns,
// which order like the values for r2 >= 0, one unsigned compare
__device__ __forceinline__ bool in_range(float r2, float rcut2) {
  return __float_as_uint(r2) - 1u < __float_as_uint(rcut2) - 1u;
}
__device__ __forceinline__ bool in_range(double r2, double rcut2) { return r2 < rcut2 && r2 > 0.0; }

// force of one entry at offset (dx, dy, dz), 0 < r^2 < r_cut^2 (the caller
// has tested the range)
template <class R>
__device__ __forceinline__ void pair_force(R dx, R dy, R dz, R r2, R m, const R* hep, R hi, R hmax,
                                           const WalkConst<R>& C, R& ax, R& ay, R& az) {
  R r, ir;
  inv_and_r(r2, r, ir);
  R fac = ir * ir * ir;
  // the entry's spline radius is read only when some softening of this step
  // reaches r (hmax: the largest radius of any particle or node)
  if (r < hmax) {
    const R he = *hep, h = he > hi ? he : hi;
    if (r < h) {
      if (sizeof(R) == 4)
        fac = (R)spline_fac_ir((float)r, (float)ir, (float)h);
      else
        fac = spline_fac(r, h);
    }
  }
  R sfac;
  if (sizeof(R) == 4 && C.poly) {
    const float t = fmaf((float)r, (float)C.tcoef, -1.0f);
    float q = kSplitPoly[11];
#pragma unroll
    for (int i = 10; i >= 0; --i) q = fmaf(q, t, kSplitPoly[i]);
    sfac = (R)(ex2_approx((float)r2 * (float)C.nl2) * q);
  } else {
    sfac = split_factor(r * C.inv2rs, C.poly);
  }
  const R f = m * fac * sfac;
  ax += f * dx;
  ay += f * dy;
  az += f * dz;
}

template <class R>
__device__ __forceinline__ void pair_in_range(const LEntry<R>& E, const R* hep, const Pos<R>& P, R hi, R hmax,
                                              const WalkConst<R>& C, R& ax, R& ay, R& az) {
  R dx, dy, dz;
  const R r2 = entry_r2(E, P, dx, dy, dz);
  pair_force(dx, dy, dz, r2, E.m, hep, hi, hmax, C, ax, ay, az);
}

// Evaluate the list [0, len) for this lane's particle: the lane takes every
// Sm-th entry from `sub`.  Entries are taken 32 at a time: a cheap pass tests
// each against r_cut (and r > 0: the self pair) into a bit mask, then the lane
// evaluates only the set bits, so the force arithmetic runs for in-range pairs
// only and the warp iterates as often as its busiest lane has pairs in range.
template <class R, bool kMasked>
__device__ __forceinline__ void eval_list(const WalkSmem<R>& sm, int w, int len, int sub, int Sm, const Pos<R>& P,
                                          R hi, R hmax, const WalkConst<R>& C, R& ax, R& ay, R& az,
                                          unsigned& nin) {
  if (!kMasked) {
    // most entries in range (a group cube small against r_cut): one pass,
    // the force arithmetic guarded by the range test
    int e = sub;
    for (; e + Sm < len; e += 2 * Sm) {  // two entries per iteration (independent chains)
      const LEntry<R> E0 = sm.e[w][e], E1 = sm.e[w][e + Sm];
      R dx0, dy0, dz0, dx1, dy1, dz1;
      const R r0 = entry_r2(E0, P, dx0, dy0, dz0);
      const R r1 = entry_r2(E1, P, dx1, dy1, dz1);
      if (in_range(r0, C.rcut2)) {
        ++nin;
        pair_force(dx0, dy0, dz0, r0, E0.m, &sm.h[w][e], hi, hmax, C, ax, ay, az);
      }
      if (in_range(r1, C.rcut2)) {
        ++nin;
        pair_force(dx1, dy1, dz1, r1, E1.m, &sm.h[w][e + Sm], hi, hmax, C, ax, ay, az);
      }
    }
    if (e < len) {
      const LEntry<R> E0 = sm.e[w][e];
      R dx, dy, dz;
      const R r2 = entry_r2(E0, P, dx, dy, dz);
      if (in_range(r2, C.rcut2)) {
        ++nin;
        pair_force(dx, dy, dz, r2, E0.m, &sm.h[w][e], hi, hmax, C, ax, ay, az);
      }
    }
    return;
  }
  const int nk = sub < len ? (len - sub + Sm - 1) / Sm : 0;
  const int nkmax = __reduce_max_sync(0xffffffffu, (unsigned)nk);
  for (int kb = 0; kb < nkmax; kb += 32) {
    unsigned mask = 0;
    const int kend = nk - kb < 32 ? nk - kb : 32;
    const LEntry<R>* ep = &sm.e[w][sub + kb * Sm];
#pragma unroll 4
    for (int k = 0; k < kend; ++k) {
      R dx, dy, dz;
      const R r2 = entry_r2(ep[k * Sm], P, dx, dy, dz);
      mask |= in_range(r2, C.rcut2) ? (1u << k) : 0u;
    }
    nin += __popc(mask);
    while (__any_sync(0xffffffffu, mask != 0u)) {
      if (mask) {
        const int k = __ffs(mask) - 1;
        mask &= mask - 1u;
        const int e = sub + (kb + k) * Sm;
        pair_in_range(sm.e[w][e], &sm.h[w][e], P, hi, hmax, C, ax, ay, az);
      }
    }
  }
}

// lattice point within r_cut of the group cube (centre cg, half side hg): the
// skip rule of the node test applied to a point (its distance to the cube)
template <class R>
__device__ __forceinline__ bool near_group(uint32_t px, uint32_t py, uint32_t pz, const uint32_t (&cg)[3],
                                           uint32_t hg, const WalkConst<R>& C) {
  const uint32_t pp[3] = {px, py, pz};
  uint32_t dv[3];
  float d2f = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const uint32_t mc = (uint32_t)abs((int32_t)(pp[a] - cg[a]));
    const uint32_t dm = max(mc, hg) - hg;
    dv[a] = dm;
    d2f = fmaf((float)dm, (float)dm, d2f);
  }
  if (d2f <= C.skip_lo) return true;
  if (d2f >= C.skip_hi) return false;
  return exact_d2(dv) <= C.skip_d2;
}

template <class R>
__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

__device__ __forceinline__ unsigned long long radius_bits(float v) { return __float_as_uint(v); }
__device__ __forceinline__ unsigned long long radius_bits(double v) { return (unsigned long long)__double_as_longlong(v); }
template <class R>
__device__ __forceinline__ R radius_of(unsigned long long b);
template <>
__device__ __forceinline__ float radius_of<float>(unsigned long long b) { return __uint_as_float((unsigned)b); }
template <>
__device__ __forceinline__ double radius_of<double>(unsigned long long b) { return __longlong_as_double((long long)b); }

// per-step walk inputs: packed particle entries (position, G m / s^2) and spline
// radius, node spline radius
template <class R>
__global__ void k_walk_prep(const int32_t* __restrict__ d_n, int64_t cap, const uint32_t* __restrict__ u,
                            const uint32_t* __restrict__ k, const int32_t* __restrict__ lvl,
                            const Node* __restrict__ nodes, Entry<R>* __restrict__ pm,
                            R* __restrict__ ph, R* __restrict__ nh, R gm0, R h0,
                            unsigned long long* __restrict__ hmax_bits) {
  const int64_t n = *d_n;
  int64_t nn = 0;
  for (int j = 0; j <= kMaxLevel; ++j) nn += lvl[j];
  const int64_t m = n > nn ? n : nn;
  uint32_t kbig = 1;  // largest multiplicity seen (radius h0 k^(1/3) grows with it)
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n) {
      uint32_t kk = k[i];
      Entry<R> E;  // packed: one vector load per particle the walk lists
      E.x = u[i];
      E.y = u[cap + i];
      E.z = u[2 * cap + i];
      E.m = gm0 * (R)kk;
      pm[i] = E;
      ph[i] = kk == 1 ? h0 : h0 * cbrt((R)kk);
      kbig = max(kbig, kk);
    }
    if (i < nn) {
      uint32_t km = nodes[i].kmax;
      nh[i] = km == 1 ? h0 : h0 * cbrt((R)km);
      kbig = max(kbig, km);
    }
  }
  kbig = __reduce_max_sync(0xffffffffu, kbig);
  if ((threadIdx.x & 31) == 0 && kbig > 1) {
    const R hb = h0 * cbrt((R)kbig);  // the same expression as the radii above
    atomicMax(hmax_bits, radius_bits(hb));
  }
}

// frontier table: every node of depth f, and every leaf above it, writes its
// index into the depth-f cells it covers (cells partition the box: no conflicts)
__global__ void k_front_fill(const int32_t* __restrict__ lvl, const Node* __restrict__ nodes, int f,
                             int32_t* __restrict__ ftab) {
  int64_t nf = 0;
  for (int j = 0; j <= f; ++j) nf += lvl[j];
  const int D = 1 << f;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nf; t += (int64_t)gridDim.x * blockDim.x) {
    const Node nd = nodes[t];
    const int j = (int)(nd.meta & 0xff);
    if (j < f && nd.child >= 0) continue;  // internal above f: its depth-f descendants write
    const int span = 1 << (f - j);
    const uint32_t h = j == 0 ? 0x80000000u : (1u << (31 - j));
    const int x0 = (int)((nd.cx - h) >> (32 - f)), y0 = (int)((nd.cy - h) >> (32 - f)),
              z0 = (int)((nd.cz - h) >> (32 - f));
    for (int a = 0; a < span; ++a)
      for (int b = 0; b < span; ++b)
        for (int c = 0; c < span; ++c) ftab[((int64_t)(x0 + a) * D + (y0 + b)) * D + (z0 + c)] = (int32_t)t;
  }
}

// window frontier table at depth F > f: every node of depth F, and every leaf
// above it, writes its index into the depth-F cells it covers, with F - depth
// and a flag for an ancestor at depths [f, F) that some group might accept.
// An ancestor a is "always opened" when every group cube within r_cut of its
// cube opens it: the COM distance to any such group cube is at most
// sqrt(skip_d2) + (distance from the COM to the farthest corner of a's cube),
// and that passes the open test of a's depth.  Below always-opened ancestors
// the per-group walk reaches exactly the depth-F nodes within r_cut.
// far2max[l]: largest squared COM-to-farthest-corner distance of a depth-l
// node that is always opened, (sqrt(open_d2[l]) - sqrt(skip_d2))^2 shrunk by a
// relative 2^-12 so that the FP32 sum below decides on the safe side (-1:
// never; +inf: the threshold opens at every distance)
struct FarMax {
  float v[kMaxLevel + 1];
};
__global__ void k_front_fill_F(const int32_t* __restrict__ lvl, const Node* __restrict__ nodes,
                               const int32_t* __restrict__ parent, int f, int F, FarMax far2max,
                               int32_t* __restrict__ ftab, uint8_t* __restrict__ fspan) {
  int64_t nF = 0;
  for (int j = 0; j <= F; ++j) nF += lvl[j];
  const int D = 1 << F;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nF; t += (int64_t)gridDim.x * blockDim.x) {
    const Node nd = nodes[t];
    const int j = (int)(nd.meta & 0xff);
    if (j < F && nd.child >= 0) continue;  // internal above F: its depth-F descendants write
    bool may_accept = false;
    for (int32_t a = parent[t]; a >= 0; a = parent[a]) {
      const Node an = nodes[a];
      const int ja = (int)(an.meta & 0xff);
      if (ja < f) break;  // above f no node is ever accepted
      const float ha = (float)(1u << (31 - ja));
      float far2 = 0.f;
      const uint32_t cm[3] = {an.comx, an.comy, an.comz}, cn[3] = {an.cx, an.cy, an.cz};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float d = (float)abs((int32_t)(cm[q] - cn[q])) + ha;
        far2 = fmaf(d, d, far2);
      }
      if (!(far2 <= far2max.v[ja])) may_accept = true;
    }
    const int span = 1 << (F - j);
    const uint32_t h = j == 0 ? 0x80000000u : (1u << (31 - j));
    const int x0 = (int)((nd.cx - h) >> (32 - F)), y0 = (int)((nd.cy - h) >> (32 - F)),
              z0 = (int)((nd.cz - h) >> (32 - F));
    const uint8_t sp = (uint8_t)((F - j) | (may_accept ? 0x80 : 0));
    for (int a = 0; a < span; ++a)
      for (int b = 0; b < span; ++b)
        for (int c = 0; c < span; ++c) {
          const int64_t cell = ((int64_t)(x0 + a) * D + (y0 + b)) * D + (z0 + c);
          ftab[cell] = (int32_t)t;
          fspan[cell] = sp;
        }
  }
}

// kMasked: evaluate lists with the range-masked pass (pays off when many
// listed entries lie beyond r_cut of a given particle: groups not small
// against r_cut), else with one range-guarded pass.  kDiag: also count node
// tests, traversal rounds and the deepest stack use (three instructions per
// round, ~1.5% of the walk: only while asked for)
template <class R, bool kMasked, bool kDiag>
__global__ void __launch_bounds__(kWarps * 32, sizeof(R) == 4 ? 8 : 5) k_walk(
    const int32_t* __restrict__ groups, const uint64_t* __restrict__ counters, unsigned int* __restrict__ next,
    const Node* __restrict__ nodes, const R* __restrict__ nh, int64_t cap, const uint32_t* __restrict__ u,
    const Entry<R>* __restrict__ pm, const R* __restrict__ ph, R* __restrict__ p, R* __restrict__ g, WalkConst<R> C,
    uint32_t* __restrict__ err, unsigned long long* __restrict__ pairs, int32_t* __restrict__ wlen) {
  extern __shared__ unsigned char smem_raw[];
  WalkSmem<R>& sm = *reinterpret_cast<WalkSmem<R>*>(smem_raw);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t ngroups = (int64_t)counters[2];
  unsigned npairs = 0;  // listed pairs of this warp (lane 0 counts them; < 2^32 per warp)
  unsigned nin = 0;               // pairs in range (0 < r < r_cut) evaluated by this lane
  int maxtop = 0;  // deepest stack use of this warp (diagnostic)
  unsigned ntests = 0, nrounds = 0;  // node tests and traversal rounds of this warp (diagnostic)
  unsigned nwin = 0, nfall = 0;      // group passes started from the depth-F window, and fallbacks
  // no spline radius of this step exceeds hmax (h0 unless something merged)
  const R hmax = max(C.h0, radius_of<R>(*C.hmax));
  for (;;) {
    int gi = 0;
    if (lane == 0) gi = (int)atomicAdd(next, 1u);
    gi = __shfl_sync(0xffffffffu, gi, 0);
    if ((int64_t)gi >= ngroups) break;
    const Node gn = nodes[groups[gi]];
    const int glevel = gn.meta & 0xff;
    const uint32_t hg = 1u << (31 - glevel);  // half side of the group cube
    const uint32_t cg[3] = {gn.cx, gn.cy, gn.cz};
    for (int c0 = 0; c0 < gn.count; c0 += 32) {
      const int cnt = gn.count - c0 < 32 ? gn.count - c0 : 32;
      // every lane works: lane -> particle m = lane mod cnt, the Sm lanes of
      // particle m (sub = 0 .. Sm - 1) each take every Sm-th list entry
      const int m = lane % cnt, sub = lane / cnt;
      const int Sm = 32 / cnt + (m < 32 % cnt ? 1 : 0);
      const int i = gn.start + c0 + m;
      const Pos<R> P = make_pos<R>(u[i], u[cap + i], u[2 * cap + i], cg);
      const R hi = ph[i];
      R ax = 0, ay = 0, az = 0;
      if (C.tree) {
        int top = 0, len = 0, glen = 0;
        bool started = false;
        if (C.frontF > 0 && glevel >= C.frontF - 1) {
          // the depth-F nodes (or leaves above F) of the cells within r_cut of
          // the group cube along every axis, each once (pushed from the first
          // window cell it covers), when no ancestor of theirs at depths
          // [f, F) can be accepted: the walk from f would open or skip those
          // ancestors, so the same nodes get tested
          const int F = C.frontF, shF = 32 - F;
          const uint32_t Dm = (1u << F) - 1u;
          uint32_t lo[3], na[3];
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            lo[a] = (cg[a] - hg - C.rcx - 1u) >> shF;
            const uint32_t hi = (cg[a] + hg + C.rcx) >> shF;
            na[a] = ((hi - lo[a]) & Dm) + 1u;
          }
          if (na[0] <= 6u && na[1] <= 6u && na[2] <= 6u) {
            const int nyz = (int)(na[1] * na[2]), total = (int)na[0] * nyz;
            bool bad = false;
            for (int b = 0; b < total; b += 32) {
              const int q = b + lane;
              bool push = false;
              int ni = -1;
              if (q < total) {
                const uint32_t qx = (uint32_t)(q / nyz), qr = (uint32_t)(q - (int)qx * nyz);
                const uint32_t qy = qr / na[2], qz = qr - qy * na[2];
                const uint32_t x = (lo[0] + qx) & Dm, y = (lo[1] + qy) & Dm, z = (lo[2] + qz) & Dm;
                const int64_t cell = ((int64_t)x * (Dm + 1) + y) * (Dm + 1) + z;
                ni = C.ftabF[cell];
                if (ni >= 0) {
                  const uint32_t sp = C.fspanF[cell];
                  bad = bad || (sp & 0x80u) != 0u;
                  const uint32_t e = sp & 0x7fu, sm1 = (1u << e) - 1u;
                  const bool whole = (int)e == F;  // one leaf covers the box: first window cell only
                  push = (qx == 0u || (!whole && (x & sm1) == 0u)) && (qy == 0u || (!whole && (y & sm1) == 0u)) &&
                         (qz == 0u || (!whole && (z & sm1) == 0u));
                }
              }
              const unsigned pmk = __ballot_sync(0xffffffffu, push);
              if (push) sm.stack[w][top + __popc(pmk & lt)] = ni;
              top += __popc(pmk);
            }
            started = !__any_sync(0xffffffffu, bad);
            if (!started) top = 0;
            nwin += started ? 1u : 0u;
            nfall += started ? 0u : 1u;
          }
        }
        if (started) {
        } else if (C.front > 0 && glevel >= C.front) {
          // the nodes of the 27 cells around the group's depth-f cell, each once
          const int f = C.front, D = 1 << f;
          int ni = -1;
          if (lane < 27) {
            const int x = (int)((gn.cx >> (32 - f)) + lane / 9 + D - 1) & (D - 1);
            const int y = (int)((gn.cy >> (32 - f)) + (lane / 3) % 3 + D - 1) & (D - 1);
            const int z = (int)((gn.cz >> (32 - f)) + lane % 3 + D - 1) & (D - 1);
            ni = C.ftab[((int64_t)x * D + y) * D + z];
          }
          for (int q = 0; q < 26; ++q) {
            const int o = __shfl_sync(0xffffffffu, ni, q);
            if (q < lane && o == ni) ni = -1;
          }
          const unsigned fm = __ballot_sync(0xffffffffu, ni >= 0);
          if (ni >= 0) sm.stack[w][__popc(fm & lt)] = ni;
          top = __popc(fm);
        } else {
          if (lane == 0) sm.stack[w][0] = 0;
          top = 1;
        }
        __syncwarp();
        // evaluate and empty the list (warp-uniform)
#define DZS_WALK_FLUSH()                                                     \
  do {                                                                       \
    __syncwarp();                                                            \
    eval_list<R, kMasked>(sm, w, len, sub, Sm, P, hi, hmax, C, ax, ay, az, nin); \
    if (lane == 0) npairs += (unsigned)len * (unsigned)cnt;                  \
    glen += len;                                                             \
    len = 0;                                                                 \
    __syncwarp();                                                            \
  } while (0)
        while (top > 0) {
          // the list is evaluated only here, between rounds (a round adds at
          // most 32 monopoles and the leaves that fit; the others wait)
          if (len > kList - 64) DZS_WALK_FLUSH();
          const int npop = top < 32 ? top : 32;
          if (kDiag) {
            ntests += npop;
            nrounds += 1;
          }
          int ni = lane < npop ? sm.stack[w][top - npop + lane] : -1;
          top -= npop;
          __syncwarp();
          bool acc = false, leaf = false, inner = false;
          Node nd;
          R nhi = 0;
          if (ni >= 0) {
            nd = nodes[ni];
            nhi = nh[ni];  // the node's softening, loaded beside the node
            const int nlevel = (int)(nd.meta & 0xff);
            // 32-bit gaps (half extents: group hg <= 2^31, node hn <= 2^30 below
            // the root, so hg + hn < 2^32); squared sums in FP32 decide unless
            // they fall within 2^-20 of the exact integer threshold, where the
            // uint64 sum decides -- the same decision as the integer rule
            uint32_t gp[3], dmv[3];
            float d2f = 0.f, c2f = 0.f;
            const uint32_t cm[3] = {nd.comx, nd.comy, nd.comz};
            // cube centre from the COM (inside the cube) and the level
            const uint32_t hn = 1u << (31 - nlevel), cmask = ~((hn << 1) - 1u);
            const uint32_t cn[3] = {(cm[0] & cmask) | hn, (cm[1] & cmask) | hn, (cm[2] & cmask) | hn};
            // gap = max(|dc|, h) - h; the root touches everything (h = max)
            const uint32_t h = nlevel == 0 ? 0xffffffffu : hg + (1u << (31 - nlevel));
#pragma unroll
            for (int a3 = 0; a3 < 3; ++a3) {
              const uint32_t dc = (uint32_t)abs((int32_t)(cn[a3] - cg[a3]));
              const uint32_t gap = max(dc, h) - h;
              gp[a3] = gap;
              d2f = fmaf((float)gap, (float)gap, d2f);
              const uint32_t mc = (uint32_t)abs((int32_t)(cm[a3] - cg[a3]));
              const uint32_t dm = max(mc, hg) - hg;
              dmv[a3] = dm;
              c2f = fmaf((float)dm, (float)dm, c2f);
            }
            const bool touch = (gp[0] | gp[1] | gp[2]) == 0u;
            bool keep = touch;
            if (!touch) {
              if (d2f <= C.skip_lo)
                keep = true;
              else if (d2f < C.skip_hi)
                keep = exact_d2(gp) <= C.skip_d2;
            }
            if (keep) {
              bool open = touch;
              if (!open) {
                if (c2f <= C.open_lo[nlevel])
                  open = true;
                else if (c2f < C.open_hi[nlevel])
                  open = exact_d2(dmv) <= C.open_d2[nlevel];
              }
              if (!open) {
                // an accepted monopole farther than r_cut from the group cube
                // acts on none of its particles: not listed
                acc = c2f <= C.skip_lo || (c2f < C.skip_hi && exact_d2(dmv) <= C.skip_d2);
              } else if (nd.child < 0) {
                leaf = true;
              } else {
                inner = true;
              }
            }
          }
          // accepted monopoles (at most 32 this round)
          unsigned am = __ballot_sync(0xffffffffu, acc);
          if (acc) {
            int pos = len + __popc(am & lt);
            sm.e[w][pos] = make_entry(nd.comx, nd.comy, nd.comz, C.gm0 * (R)nd.mass, cg);
            sm.h[w][pos] = nhi;
          }
          len += __popc(am);
          // children of opened inner nodes onto the stack
          // one scan for both counts: children (<= 8 per lane, total < 2^16) in
          // the low half, leaf particles (<= B <= 14 per lane) in the high half
          int nch = inner ? (int)((nd.meta >> 8) & 0xff) : 0;
          int lc = (leaf && nd.count <= C.B) ? nd.count : 0;
          const int both = warp_incl_scan<R>(nch | (lc << 16), lane);
          int ex = (both & 0xffff) - nch;
          int tot = __shfl_sync(0xffffffffu, both & 0xffff, 31);
          const int incl = both >> 16;
          if (top + tot > kStack) {
            if (lane == 0) atomicOr(err, kErrStack);
            nch = 0;
            tot = 0;
          }
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (q < nch) sm.stack[w][top + ex + q] = nd.child + q;
          top += tot;
          if (kDiag) maxtop = top > maxtop ? top : maxtop;
          // particles of opened small leaves, copied cooperatively (item t of
          // the round belongs to the lane whose inclusive end first exceeds t);
          // a particle farther than r_cut from the group cube acts on none of
          // the group's particles and is not listed
          // leaves whose particles do not fit in the list this round go back
          // on the stack (the inclusive ends grow with the lane, so the ones
          // that fit are a prefix); after the next evaluation they fit
          const int room = kList - len;
          const bool defer = lc > 0 && incl > room;
          const unsigned dm = __ballot_sync(0xffffffffu, defer);
          if (dm) {
            if (top + __popc(dm) > kStack) {
              if (lane == 0) atomicOr(err, kErrStack);
            } else if (defer) {
              sm.stack[w][top + __popc(dm & lt)] = ni;
            }
            top += top + __popc(dm) > kStack ? 0 : __popc(dm);
            if (defer) lc = 0;
          }
          // items of the leaves that stay: the largest inclusive end within
          // the room (lanes past a deferred leaf carry its items in incl)
          const int totl = (int)__reduce_max_sync(0xffffffffu, (unsigned)(incl <= room ? incl : 0));
          // item t of the owner lane is particle jbase_owner + t
          const int jbase = leaf ? nd.start - (incl - lc) : 0;
          for (int b0 = 0; b0 < totl; b0 += 32) {
            int t = b0 + lane;
            int src = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
              int v = __shfl_sync(0xffffffffu, incl, src + step - 1);
              if (v <= t) src += step;
            }
            const int jb = __shfl_sync(0xffffffffu, jbase, src);
            bool take = false;
            Entry<R> E;
            R hj = 0;
            if (t < totl) {
              const int64_t j = (int64_t)jb + t;
              E = pm[j];
              hj = ph[j];  // loaded beside the entry, before the distance test
              take = near_group(E.x, E.y, E.z, cg, hg, C);
            }
            const unsigned tm = __ballot_sync(0xffffffffu, take);
            if (take) {
              const int pos = len + __popc(tm & lt);
              sm.e[w][pos] = make_entry(E.x, E.y, E.z, E.m, cg);
              sm.h[w][pos] = hj;
            }
            len += __popc(tm);
          }
          __syncwarp();
          // big leaves (depth 21, more than B particles): stream through
          unsigned bm = __ballot_sync(0xffffffffu, leaf && nd.count > C.B);
          while (bm) {
            int src = __ffs(bm) - 1;
            bm &= bm - 1;
            int bs = __shfl_sync(0xffffffffu, nd.start, src);
            int bc = __shfl_sync(0xffffffffu, nd.count, src);
            for (int q0 = 0; q0 < bc; q0 += 32) {
              if (len + 32 > kList) DZS_WALK_FLUSH();
              bool take = false;
              Entry<R> E;
              R hj = 0;
              if (q0 + lane < bc) {
                const int64_t j = (int64_t)bs + q0 + lane;
                E = pm[j];
                hj = ph[j];
                take = near_group(E.x, E.y, E.z, cg, hg, C);
              }
              const unsigned tm = __ballot_sync(0xffffffffu, take);
              if (take) {
                const int pos = len + __popc(tm & lt);
                sm.e[w][pos] = make_entry(E.x, E.y, E.z, E.m, cg);
                sm.h[w][pos] = hj;
              }
              len += __popc(tm);
            }
            __syncwarp();
          }
        }
        DZS_WALK_FLUSH();
#undef DZS_WALK_FLUSH
        if (c0 == 0 && lane == 0) wlen[gi] = glen;
        // combine the Sm partial sums of each particle: fixed shuffle tree over
        // its lanes m, m + cnt, m + 2 cnt, ... (deterministic for a given cnt)
        const int smax = 32 / cnt + (32 % cnt ? 1 : 0);
        for (int o = 1; o < smax; o <<= 1) {
          const bool in = (sub & (2 * o - 1)) == 0 && sub + o < Sm;
          R tx = __shfl_down_sync(0xffffffffu, ax, o * cnt), ty = __shfl_down_sync(0xffffffffu, ay, o * cnt);
          R tz = __shfl_down_sync(0xffffffffu, az, o * cnt);
          if (in) {
            ax += tx;
            ay += ty;
            az += tz;
          }
        }
      }
      if (sub == 0) {
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
  unsigned long long nin64 = nin;
  for (int o = 16; o > 0; o >>= 1) nin64 += __shfl_down_sync(0xffffffffu, nin64, o);
  if (lane == 0 && npairs) atomicAdd(pairs, (unsigned long long)npairs);
  if (lane == 0 && nin64) atomicAdd(pairs + 1, nin64);
  if (kDiag && lane == 0) {
    atomicMax(pairs + 3, (unsigned long long)maxtop);
    atomicAdd(pairs + 8, (unsigned long long)ntests);
    atomicAdd(pairs + 9, (unsigned long long)nrounds);
  }
  if (lane == 0 && nwin) atomicAdd(pairs + 16, (unsigned long long)nwin);
  if (lane == 0 && nfall) atomicAdd(pairs + 17, (unsigned long long)nfall);
}

template <class R>
void walk_impl(dzs_ctx* c, bool tree, bool close_kick, int step) {
  const double s = c->scale;
  WalkConst<R> C;
  C.rcut2 = (R)((c->rcut / s) * (c->rcut / s));
  C.inv2rs = (R)(s / (2.0 * c->rs));
  C.tcoef = (R)(s / (2.0 * c->rs) * (2.0 / (double)kSplitXMax));
  C.nl2 = (R)(-1.4426950408889634 * (s / (2.0 * c->rs)) * (s / (2.0 * c->rs)));
  C.gm0 = (R)(c->gm0 / (s * s));
  C.kick = close_kick ? (R)c->T.kick2[step] : (R)0;
  C.skip_d2 = c->walk_skip_d2;
  for (int l = 0; l <= kMaxLevel; ++l) C.open_d2[l] = c->walk_open_d2[l];
  // FP32 bounds around each integer threshold: a float sum below lo is surely
  // <= T, one at or above hi surely > T (FP32 sum error < 2^-21 relative)
  auto lo_of = [](uint64_t t) { return std::nextafter((float)((double)t * (1.0 - 0x1p-20)), 0.0f); };
  auto hi_of = [](uint64_t t) { return std::nextafter((float)((double)t * (1.0 + 0x1p-20)), INFINITY); };
  C.skip_lo = lo_of(C.skip_d2);
  C.skip_hi = hi_of(C.skip_d2);
  for (int l = 0; l <= kMaxLevel; ++l) {
    C.open_lo[l] = lo_of(C.open_d2[l]);
    C.open_hi[l] = hi_of(C.open_d2[l]);
  }
  C.B = c->P.leaf_bucket;
  C.close = close_kick ? 1 : 0;
  C.tree = tree ? 1 : 0;
  C.poly = (c->P.rcut_rs / 2.0 <= (double)kSplitXMax) ? 1 : 0;
  // frontier depth: every depth above it never accepts (a non-skipped node's
  // COM distance is at most sqrt(skip_d2) + sqrt(3) l, and that opens it), and
  // its cells are wider than r_cut (cells beyond the 27 neighbours are skipped)
  C.front = 0;
  C.ftab = c->B.iscan;  // scratch: the tree's tile counts are no longer needed
  C.frontF = 0;
  C.rcx = 0;
  C.ftabF = nullptr;
  C.fspanF = nullptr;
  const int64_t ftab_cap = 2 * c->cap + 64;
  for (int f = 1; f <= 7 && ((int64_t)1 << (3 * f)) <= ftab_cap; ++f) {
    const double lf = std::ldexp(1.0, 32 - f), lp = std::ldexp(1.0, 33 - f);
    const double reach = std::sqrt((double)C.skip_d2) + 1.7320508075688772 * lp;
    // (a saturated threshold opens at every representable distance)
    const bool never = C.open_d2[f - 1] == ~0ull || reach * reach * (1.0 + 1e-9) <= (double)C.open_d2[f - 1];
    const bool wide = lf * lf > (double)C.skip_d2 * (1.0 + 1e-9);
    if (!(never && wide)) break;
    C.front = f;
  }
  // window frontier depth F (f + 2, else f + 1): the window of a group at
  // depth >= F - 1 spans at most 6 depth-F cells per axis and at most half
  // the box, and both tables fit in the scratch
  if (C.front > 0 && tree) {
    uint64_t r = (uint64_t)std::sqrt((double)C.skip_d2);
    while (r * r > C.skip_d2) --r;
    while ((r + 1) * (r + 1) <= C.skip_d2) ++r;
    const int64_t cells_f = (int64_t)1 << (3 * C.front);
    for (int F = C.front + 2; F > C.front; --F) {
      if (F > kMaxLevel || r >= (1ull << 30)) continue;
      const int64_t cells = (int64_t)1 << (3 * F);
      const int64_t off = (cells_f + 3) & ~(int64_t)3;
      if (off + cells + (cells + 3) / 4 > ftab_cap) continue;
      const uint64_t sF = 1ull << (32 - F);
      const uint64_t npts = 2 * sF + 2 * r + 2;  // lattice points of the widest window (inclusive)
      const uint64_t nmax = (npts - 1) / sF + 2;
      if (nmax > 6 || 2 * nmax > (1ull << F)) continue;
      C.frontF = F;
      C.rcx = (uint32_t)r;
      C.ftabF = c->B.iscan + off;
      C.fspanF = (const uint8_t*)(c->B.iscan + off + cells);
      break;
    }
  }
  Entry<R>* pm = (Entry<R>*)c->B.wpm;
  R* ph = (R*)c->B.wph;
  R* nh = (R*)c->B.wnh;
  C.h0 = (R)(2.8 * c->eps0 / s);
  unsigned long long* hmax_slot = (unsigned long long*)(c->B.counters + 24);
  C.hmax = hmax_slot;
  cudaMemsetAsync(hmax_slot, 0, sizeof(uint64_t), c->stream);
  k_walk_prep<R><<<grid_for(c->node_cap), kThreads, 0, c->stream>>>(c->B.n, c->cap, c->B.u, c->B.k, c->B.lvl_count,
                                                                     c->B.nodes, pm, ph, nh, C.gm0, C.h0, hmax_slot);
  if (C.front > 0 && tree) {
    const int64_t cells = (int64_t)1 << (3 * C.front);
    c->launches += 1;
    cudaMemsetAsync(c->B.iscan, 0xff, sizeof(int32_t) * cells, c->stream);
    k_front_fill<<<grid_for(cells, kThreads, 4), kThreads, 0, c->stream>>>(c->B.lvl_count, c->B.nodes, C.front,
                                                                               c->B.iscan);
    if (C.frontF > 0) {
      const int64_t cellsF = (int64_t)1 << (3 * C.frontF);
      c->launches += 1;
      cudaMemsetAsync((void*)C.ftabF, 0xff, sizeof(int32_t) * cellsF, c->stream);
      cudaMemsetAsync((void*)C.fspanF, 0, (size_t)cellsF, c->stream);
      FarMax fm;
      const double skip_r = std::sqrt((double)C.skip_d2) * (1.0 + 1e-12);
      for (int l = 0; l <= kMaxLevel; ++l) {
        if (C.open_d2[l] == ~0ull) {
          fm.v[l] = INFINITY;
          continue;
        }
        const double room = std::sqrt((double)C.open_d2[l]) * (1.0 - 1e-12) - skip_r;
        fm.v[l] = room > 0.0 ? (float)(room * room * (1.0 - 0x1p-12)) : -1.0f;
      }
      k_front_fill_F<<<grid_for(cellsF, kThreads, 4), kThreads, 0, c->stream>>>(
          c->B.lvl_count, c->B.nodes, c->B.parent, C.front, C.frontF, fm, (int32_t*)C.ftabF, (uint8_t*)C.fspanF);
    }
  }
  // automatic: the range-masked evaluation when the walk groups of a uniform
  // particle set (leaves of ~B particles, side ~2 spacings) are at least
  // r_cut / 2 wide; both evaluate the same pairs in the same order
  const double spacing = c->P.box / c->P.n1d;
  const bool masked = c->P.walk_eval == DZS_WALK_MASKED ||
                      (c->P.walk_eval == DZS_WALK_AUTO && 4.0 * spacing >= c->rcut);
  const bool diag = c->walk_diag;
  auto kern = masked ? (diag ? k_walk<R, true, true> : k_walk<R, true, false>)
                     : (diag ? k_walk<R, false, true> : k_walk<R, false, false>);
  size_t sm = sizeof(WalkSmem<R>);
  static bool attr_done[2][2][2] = {};
  if (!attr_done[sizeof(R) == 8][masked][diag]) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr_done[sizeof(R) == 8][masked][diag] = true;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarps * 32, sm);
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->dev);
  int grid = (per_sm > 0 ? per_sm : 1) * (nsm > 0 ? nsm : 1);
  unsigned int* next = (unsigned int*)(c->B.counters + 6);
  cudaMemsetAsync(next, 0, sizeof(unsigned int), c->stream);
  kern<<<grid, kWarps * 32, sm, c->stream>>>(c->B.groups, c->B.counters, next, c->B.nodes, nh, c->cap, c->B.u,
                                                  pm, ph, (R*)c->B.p, (R*)c->B.g, C, c->B.err,
                                                  (unsigned long long*)(c->B.counters + 4), c->B.wlen);
}

}  // namespace

void launch_walk(dzs_ctx* c, bool tree, bool close_kick, int step) {
  c->launches += 2;
  if (c->fp64)
    walk_impl<double>(c, tree, close_kick, step);
  else
    walk_impl<float>(c, tree, close_kick, step);
}

}  // namespace dzs
