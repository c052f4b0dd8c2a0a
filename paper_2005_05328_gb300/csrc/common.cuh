// common.cuh -- shared device helpers and the context layout of the DZS
// TreePM library (paper: Garaldi, Nori & Baldi, arXiv 2005.05328).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "dzs.h"

namespace dzs {

constexpr int kThreads = 256;
constexpr int kMaxLevel = 21;  // 21 Morton bits per axis

// device error word bits (never a trap: kernels record and skip)
enum : uint32_t {
  kErrNodes = 1u,    // tree node capacity exceeded
  kErrStack = 2u,    // walk stack overflow
  kErrRing = 4u,     // lightcone ring full (records dropped)
  kErrGroups = 8u,   // group capacity exceeded
  kErrSort = 16u,    // inconsistent radix sort histogram
  kErrCell = 32u,    // CIC cell start table inconsistent
};

// flag bits: bit 0 crossed (public), bit 1 merged (public), bit 2 crossed in
// the current step (transient: cleared by the next opening kick)
constexpr uint8_t kFlCrossed = 1, kFlMerged = 2, kFlNow = 4;

__host__ __device__ inline uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x1fffffu;
  x = (x | (x << 32)) & 0x1f00000000ffffull;
  x = (x | (x << 16)) & 0x1f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

// 63-bit Morton key of the top 21 bits per axis; x takes the highest bit of
// each 3-bit digit, so key >> 3(21 - j) is the octree cell at depth j
__host__ __device__ inline uint64_t morton_key(uint32_t x, uint32_t y, uint32_t z) {
  return (spread3(x >> 11) << 2) | (spread3(y >> 11) << 1) | spread3(z >> 11);
}

// squared lattice distance to the observer at 2^31 (exact, < 3 * 2^62)
__host__ __device__ inline uint64_t dist2_obs(uint32_t x, uint32_t y, uint32_t z) {
  int64_t a = (int32_t)(x - 0x80000000u), b = (int32_t)(y - 0x80000000u), c = (int32_t)(z - 0x80000000u);
  return (uint64_t)(a * a) + (uint64_t)(b * b) + (uint64_t)(c * c);
}

template <class R>
struct cplx {
  R x, y;
};

template <class R>
__device__ __forceinline__ cplx<R> cmul(cplx<R> a, cplx<R> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// streaming multiprocessors of the current device (queried once per device)
int sm_count();

// blocks for n items: one per `threads` items, at most `per_sm` per SM
inline int grid_for(int64_t n, int threads = kThreads, int per_sm = 16) {
  const int64_t cap = (int64_t)per_sm * sm_count();
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  return (int)(b < cap ? b : cap);
}

// ---------------------------------------------------------------- context

struct Tables {
  std::vector<double> a, drift, kick1, kick2, rlc;
  std::vector<uint64_t> rlat;
  double dplus_i = 0, f_i = 0, e_i = 0, power_amp = 0;
};

// node record of the oct-tree, 48 bytes
// the first 32 bytes hold what the tree walk reads per node test (the cube
// centre follows from the COM, which lies in the cube, and the level)
struct Node {
  uint32_t comx, comy, comz;  // rounded integer centre of mass
  uint32_t mass;              // sum of k
  int32_t start, count;       // particle range
  int32_t child;              // first child, -1 for a leaf
  uint32_t meta;              // level (bits 0-7) | nchild (bits 8-15)
  uint32_t cx, cy, cz;        // cube centre (lattice)
  uint32_t kmax;              // largest member k (softening)
};
static_assert(sizeof(Node) == 48, "node layout");

struct Buffers {
  // particle state (primary and alternate for permutations / compaction)
  uint32_t *u = nullptr, *u2 = nullptr;  // [3][cap]
  void *p = nullptr, *p2 = nullptr;      // real [3][cap]
  void* g = nullptr;                     // real [3][cap]
  void* gsave = nullptr;                 // real [3][cap] (accelerations kept across dzs_accel)
  uint32_t *k = nullptr, *k2 = nullptr, *id = nullptr, *id2 = nullptr;
  uint8_t *fl = nullptr, *fl2 = nullptr;
  // sort
  uint64_t *key = nullptr, *key2 = nullptr;
  uint32_t *idx = nullptr, *idx2 = nullptr;
  uint32_t* hist = nullptr;  // [256][max blocks]
  // generic scan scratch
  int64_t* blocksum = nullptr;
  int32_t* iscan = nullptr;  // [cap + 1]
  // merge
  uint64_t* prefix = nullptr;  // [4][cap + 1]: sum k, sum k ux, uy, uz
  int32_t* mend = nullptr;     // [cap]
  // tree
  Node* nodes = nullptr;
  int32_t* lvl_count = nullptr;  // [kMaxLevel + 2]
  int32_t* cfirst = nullptr;     // [node cap] first-child index of each node (tree build)
  int32_t* parent = nullptr;     // [node cap] parent node (-1 at the root)
  void* cicw = nullptr;          // real [8][cap] CIC corner weight sums per mesh cell (deposit)
  int32_t* groups = nullptr;     // [cap]
  void* wpm = nullptr;           // real [cap]: G m / s^2 per particle (walk, lattice units)
  void* wph = nullptr;           // real [cap]: spline radius per particle (lattice units)
  void* wnh = nullptr;           // real [node cap]: node spline radius (lattice units)
  int32_t* wlen = nullptr;       // [cap]: interaction-list length of each walk group (last walk)
  int32_t* group_head = nullptr; // [cap]
  // PM
  void* rho = nullptr;    // real [M^3]
  void* spec = nullptr;   // cplx [M][M][M/2+1]
  void* phi = nullptr;    // real [M^3]
  int32_t* cell_start = nullptr;  // [M^3 + 1]
  void* twiddle = nullptr;        // cplx tables
  void* green_axis = nullptr;     // per-axis Green factors
  // lightcone ring
  dzs_lc_record* ring = nullptr;
  // device scalars
  int32_t* n = nullptr;          // particle count
  uint32_t* err = nullptr;       // error word
  // [32]: 0 ring head, 1 records dropped, 2 groups, 3 nodes, 4 listed pairs
  // (list entries x group particles), 5 in-range pairs (0 < r < r_cut),
  // 6 walk work counter, 7 deepest walk stack, 8..11 diagnostics integer sums,
  // 12 walk node tests, 13 walk rounds, 14 a_min^2, 15 scratch, 16 walk units,
  // 18 crossings of the next step (ring check)
  uint64_t* counters = nullptr;
  double* diag = nullptr;        // [8 + blocks] diagnostics partials
  void* convert = nullptr;       // double [3][cap] conversion scratch
};

// where lightcone records are binned (sky map, 3D lightcone); null: nowhere
struct ObserveTarget {
  unsigned long long* sky = nullptr;   // [12 nside^2] mass per RING pixel, or null
  unsigned long long* grid = nullptr;  // [mesh^3] NGP mass of crossing positions, or null
  int64_t nside = 0, mesh = 0;
  double a_lo = 0, a_hi = 0;           // records with a_lo <= a* < a_hi
  double half = 0, box = 0;            // observer at (L/2, L/2, L/2)
};

}  // namespace dzs

struct dzs_ctx {
  dzs_params P;
  int dev = 0;
  cudaStream_t stream = nullptr;
  bool fp64 = false;
  int64_t N0 = 0, cap = 0, node_cap = 0;
  int M = 0, logM = 0, n1 = 0;  // logM: depth of the Morton cell table (floor log2 M)
  bool mesh_pow2 = true;         // false: M = 3 2^a, deposited through a row-major cell sort
  int sort_blocks = 0;
  double lat = 0, scale = 0, gm0 = 0, eps0 = 0, rs = 0, rcut = 0, rcut_lat2 = 0;
  int jmin = 1;
  uint64_t blat = 0;
  uint64_t merge_thr[dzs::kMaxLevel + 1];
  // exact integer forms of the walk's FP64 skip and open comparisons
  uint64_t walk_skip_d2 = 0;
  uint64_t walk_open_d2[dzs::kMaxLevel + 1];
  dzs::Tables T;
  int32_t step = 0;
  bool have_state = false;
  bool poisoned = false;
  // dynamical DZS criterion: g is in the particles' current order (false
  // between a step's sort and its force stage), and a_min^2 of this step
  // has been reduced into counters[14] (after the kick-drift stage)
  bool g_aligned = true;
  bool amin2_ready = false;
  uint64_t drained = 0;
  size_t ring_cap = 0;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  dzs::Buffers B;
  dzs::ObserveTarget obs;  // device buffers owned by the context (dzs_observe_enable)
  void* sht_work = nullptr;  // harmonic-analysis scratch (dzs_skymap_alm)
  size_t sht_bytes = 0;
  std::string err;
  uint64_t launches = 0;  // kernels launched (host-side count)
  // per-stage CUDA-event profiling
  bool prof_on = false;
  bool walk_diag = false;  // count the walk's node tests, rounds and stack depth
  struct ProfEv {
    int cat;
    cudaEvent_t a, b;
  };
  std::vector<ProfEv> prof_pending;
  std::vector<cudaEvent_t> ev_pool;
  double prof_ms[8] = {0};
  uint64_t prof_calls[8] = {0};
  // pipelined per-step results (dzs_pipeline): the last kPipe steps' diagnostics,
  // ring head, dropped count and error word in pinned host memory, each slot
  // written by copies enqueued at the end of its step and closed by an event
  static constexpr int kPipe = 4;
  struct PipeSlot {
    double diag[8];
    uint64_t ring[2];  // records written so far, dropped so far
    uint32_t err[4];
  };
  bool pipe_on = false;
  PipeSlot* pipe = nullptr;  // [kPipe], pinned
  cudaEvent_t pipe_ev[kPipe] = {nullptr, nullptr, nullptr, nullptr};
  int32_t pipe_step[kPipe] = {-1, -1, -1, -1};  // completed-step count each slot holds
  cudaStream_t copy_stream = nullptr;          // record copies beside the compute stream
};

namespace dzs {

// host-side cosmology (host.cu)
void compute_tables(const dzs_params& P, Tables& T);
double bbks_shape(const dzs_params& P, double k);  // k^ns T(k)^2

// launchers (each file); all enqueue on c->stream
void launch_kick_drift(dzs_ctx* c, int step, bool kick, bool drift);
void launch_records(dzs_ctx* c, int step);
void launch_count_crossings(dzs_ctx* c, int step, unsigned long long* count);
void launch_twin_displacement(dzs_ctx* a, dzs_ctx* b, int32_t* map, const double* edges, int nbins, double h,
                              unsigned long long* counts, unsigned long long* stats);
void launch_sort(dzs_ctx* c);
void launch_sort_keys(dzs_ctx* c, uint64_t* ka, uint64_t* kb, uint32_t* va, uint32_t* vb, int passes);
void launch_keys(dzs_ctx* c);
void launch_unpermute(dzs_ctx* c, double* g_out);
void launch_close_kick(dzs_ctx* c, int step);
void launch_merge(dzs_ctx* c, uint64_t rlat);
// exclusive uint64 prefix sums of k, k ux, k uy, k uz over the particles into
// B.prefix ([4][cap + 1])
void launch_mass_prefix(dzs_ctx* c);
void launch_amin2(dzs_ctx* c);
void launch_tree(dzs_ctx* c);
void launch_cell_start(dzs_ctx* c);
void launch_pm_deposit(dzs_ctx* c);
void launch_pm_fft(dzs_ctx* c);
void launch_pm_interp(dzs_ctx* c);
void launch_walk(dzs_ctx* c, bool tree, bool close_kick, int step);
void launch_diagnostics(dzs_ctx* c);
void launch_ics(dzs_ctx* c);
void launch_to_double(dzs_ctx* c, const void* src, int64_t count, double* dst);
void launch_from_double(dzs_ctx* c, const double* src, int64_t count, void* dst);
void launch_fft_init(dzs_ctx* c);
void launch_pk(dzs_ctx* c, int nbins, double* d_part, double* d_out, double shot);
void launch_fof(dzs_ctx* c, int depth, uint64_t T, int nmin, int64_t* d_label, dzs_halo** d_halos);
void launch_sum_k2(dzs_ctx* c, unsigned long long* out);
void launch_observe_records(dzs_ctx* c, const dzs_lc_record* d_rec, int64_t n);
size_t sht_work_bytes(int64_t nside, int lmax);
size_t sht_shared_bytes(int lmax);
void launch_sht(dzs_ctx* c, int lmax, void* work, double2** d_alm, double** d_cl);
void upload_fft_constants(int dev);  // register-FFT twiddles, once per device
template <class R>
void fft_r2c_3d(dzs_ctx* c, const R* in, cplx<R>* out, int n, const cplx<R>* tw);
template <class R>
void fft_c2r_3d(dzs_ctx* c, cplx<R>* in, R* out, int n, const cplx<R>* tw, const R* green, R gfac);

// deterministic exclusive scan of int32 flags/counts -> iscan[0..n], n on device
void exclusive_scan_i32(dzs_ctx* c, const int32_t* in, int32_t* out, const int32_t* d_n, int64_t cap);

}  // namespace dzs
