// api.cu -- the C ABI of include/dzs.h: context life cycle, state injection
// and extraction, the stage runner of one KDK step, lightcone drain and
// diagnostics.  Step order (paper Sec. 2.2: DZS on global steps, tree rebuilt
// and forces recomputed after a merge): opening kick + drift + crossing ->
// records -> Morton sort -> merge -> tree -> PM -> walk + closing kick.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <atomic>

#include "common.cuh"

using namespace dzs;

namespace {

thread_local std::string g_create_error;

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

int ilog2i(int64_t v) {
  int l = 0;
  while ((1ll << l) < v) ++l;
  return l;
}

const char* validate(const dzs_params* p) {
  if (!p) return "params is NULL";
  auto pow2_or_3pow2 = [](int64_t v) { return is_pow2(v) || (v % 3 == 0 && is_pow2(v / 3)); };
  if (!pow2_or_3pow2(p->n1d) || p->n1d < 2 || p->n1d > 512) return "n1d must be 2^a or 3 2^a in [2, 512]";
  if (!pow2_or_3pow2(p->mesh) || p->mesh < 8 || p->mesh > 512 || p->mesh % 8 != 0)
    return "mesh must be 2^a or 3 2^a, a multiple of 8, in [8, 512]";
  if (!(p->box > 0)) return "box must be positive";
  if (!(p->omega_m > 0) || !(p->omega_l >= 0)) return "omega_m > 0 and omega_l >= 0 required";
  if (!(p->hubble > 0) || !(p->sigma8 >= 0)) return "hubble > 0 and sigma8 >= 0 required";
  if (!(p->z_init > 0)) return "z_init must be positive";
  if (p->nsteps < 1 || p->nsteps > 100000) return "nsteps out of range";
  if (p->leaf_bucket < 1 || p->leaf_bucket > 14) return "leaf_bucket must be in [1, 14]";
  if (p->walk_group < p->leaf_bucket || p->walk_group > 64) return "walk_group must be in [leaf_bucket, 64]";
  if (p->merge_level < 1 || (1 << (p->merge_level - 1)) > p->n1d) return "merge_level out of range";
  if (!(p->rs_cells > 0) || !(p->rcut_rs > 0)) return "rs_cells and rcut_rs must be positive";
  if (!(p->theta > 0)) return "theta must be positive";
  if (!(p->soft_frac > 0)) return "soft_frac must be positive";
  if (!(p->theta_dzs > 0)) return "theta_dzs must be positive";
  if (!(p->buffer_cells >= 0)) return "buffer_cells must be >= 0";
  if (p->rlc_mode != DZS_RLC_SWEEP && p->rlc_mode != DZS_RLC_PHYSICAL) return "unknown rlc_mode";
  if (p->precision != DZS_FP32 && p->precision != DZS_FP64) return "unknown precision";
  if (p->dzs_criterion != DZS_CRIT_GEOMETRIC && p->dzs_criterion != DZS_CRIT_DYNAMICAL) return "unknown dzs_criterion";
  if (!(p->alpha_dyn >= 0)) return "alpha_dyn must be >= 0";
  if (p->walk_eval < DZS_WALK_AUTO || p->walk_eval > DZS_WALK_GUARDED) return "walk_eval must be 0, 1 or 2";
  if (p->capacity > (uint64_t)p->n1d * p->n1d * p->n1d) return "capacity exceeds n1d^3";
  return nullptr;
}

// largest x in [0, 2^64) with pass(x) true, for a predicate that is true on a
// prefix of the integers (pass(0) must hold)
template <class F>
uint64_t largest_passing(F pass) {
  uint64_t lo = 0, hi = ~0ull;
  if (pass(hi)) return hi;
  while (hi - lo > 1) {
    uint64_t mid = lo + (hi - lo) / 2;
    if (pass(mid))
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

struct Layout {
  size_t total = 0;
  size_t take(size_t bytes) {
    size_t off = total;
    total += (bytes + 255) & ~size_t(255);
    return off;
  }
};

// offsets of every device buffer in the arena (also used for the footprint)
struct Plan {
  int64_t cap, node_cap, m3, nspec, nb, nchunks, ring;
  size_t rsz;
  size_t o_u, o_u2, o_p, o_p2, o_g, o_gsave, o_k, o_k2, o_id, o_id2, o_fl, o_fl2, o_key, o_key2, o_idx, o_idx2, o_hist,
      o_blocksum, o_iscan, o_prefix, o_mend, o_nodes, o_lvl, o_cfirst, o_parent, o_cicw, o_groups, o_ghead, o_wpm, o_wph, o_wnh, o_wlen,
      o_rho, o_spec, o_phi,
      o_cstart, o_tw, o_green, o_ring, o_n, o_err, o_counters, o_diag, o_convert;
  size_t total;
  explicit Plan(const dzs_params& P) {
    cap = P.capacity ? (int64_t)P.capacity : (int64_t)P.n1d * P.n1d * P.n1d;
    node_cap = 2 * cap + 1024;
    m3 = (int64_t)P.mesh * P.mesh * P.mesh;
    nspec = (int64_t)P.mesh * P.mesh * (P.mesh / 2 + 1);
    nb = (cap + 1023) / 1024;  // digit-histogram tiles: enough for sort tiles of >= 1024 keys
    nchunks = (cap + 1024) / 1024 + 1;
    ring = P.lc_capacity ? (int64_t)P.lc_capacity : cap;
    rsz = P.precision == DZS_FP64 ? 8 : 4;
    Layout L;
    o_u = L.take(12 * cap);
    o_u2 = L.take(12 * cap);
    o_p = L.take(3 * rsz * cap);
    o_p2 = L.take(3 * rsz * cap);
    o_g = L.take(3 * rsz * cap);
    o_gsave = L.take(3 * rsz * cap);
    o_k = L.take(4 * cap);
    o_k2 = L.take(4 * cap);
    o_id = L.take(4 * cap);
    o_id2 = L.take(4 * cap);
    o_fl = L.take(cap);
    o_fl2 = L.take(cap);
    o_key = L.take(8 * cap);
    o_key2 = L.take(8 * cap);
    o_idx = L.take(4 * cap);
    o_idx2 = L.take(4 * cap);
    o_hist = L.take(4 * (257 * nb + 256));
    o_blocksum = L.take(8 * 4 * (nchunks + 2));
    o_iscan = L.take(4 * (2 * cap + 64));  // also the tree's per-tile counts (23 per 1024 particles)
    o_prefix = L.take(8 * 4 * (cap + 1));
    o_mend = L.take(4 * cap);
    o_nodes = L.take(sizeof(Node) * node_cap);
    o_lvl = L.take(4 * 32);
    o_cfirst = L.take(4 * node_cap);
    o_parent = L.take(4 * node_cap);
    o_cicw = L.take(8 * rsz * cap);
    o_groups = L.take(4 * cap);
    o_ghead = L.take(4 * cap);
    o_wpm = L.take((rsz == 8 ? 24 : 16) * cap);  // packed walk entries: lattice position, G m
    o_wph = L.take(rsz * cap);
    o_wnh = L.take(rsz * node_cap);
    o_wlen = L.take(4 * cap);
    o_rho = L.take(rsz * m3);
    o_spec = L.take(2 * rsz * nspec);
    o_phi = L.take(rsz * m3);
    o_cstart = L.take(4 * (m3 + 1));
    o_tw = L.take(2 * rsz * (P.mesh / 2 + 1));
    o_green = L.take(rsz * (2 * P.mesh + 1));
    o_ring = L.take(sizeof(dzs_lc_record) * ring);
    o_n = L.take(16);
    o_err = L.take(16);
    o_counters = L.take(8 * 32);
    o_diag = L.take(8 * (8 + 3 * 304));
    o_convert = L.take(8 * 3 * cap);
    total = L.total;
  }
};

#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) return fail(c, DZS_ECUDA, #call, cudaGetErrorString(e_)); \
  } while (0)

// host-side allocation-failure injection (tests): the k-th device
// allocation from now on fails as if the device were out of memory
std::atomic<int> g_fail_alloc{0};

cudaError_t dev_alloc(void** ptr, size_t bytes) {
  int k = g_fail_alloc.load();
  while (k > 0) {
    if (g_fail_alloc.compare_exchange_weak(k, k - 1)) {
      if (k == 1) return cudaErrorMemoryAllocation;
      break;
    }
  }
  return cudaMalloc(ptr, bytes);
}

dzs_status fail(dzs_ctx* c, dzs_status s, const char* what, const char* detail = nullptr) {
  std::string m = what ? what : "";
  if (detail) m += std::string(": ") + detail;
  if (c) {
    c->err = m;
    if (s == DZS_EDEVICE || s == DZS_ETIMEOUT) c->poisoned = true;
  } else {
    g_create_error = m;
  }
  return s;
}

dzs_status check_device_errors(dzs_ctx* c) {
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(c, DZS_EDEVICE, "device failure", cudaGetErrorString(e));
  uint32_t err = 0;
  e = cudaMemcpy(&err, c->B.err, sizeof(uint32_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(c, DZS_EDEVICE, "device failure", cudaGetErrorString(e));
  if (err & (kErrNodes | kErrStack | kErrGroups)) {
    char buf[160];
    snprintf(buf, sizeof buf, "device buffer overflow (error word 0x%x)", err);
    return fail(c, DZS_EOVERFLOW, buf);
  }
  return DZS_OK;
}

dzs_status guard(dzs_ctx* c) {
  if (!c) return DZS_EINVAL;
  if (c->poisoned) return fail(c, DZS_ESTATE, "context poisoned by an earlier device failure");
  cudaError_t e = cudaSetDevice(c->dev);
  if (e != cudaSuccess) return fail(c, DZS_ECUDA, "cudaSetDevice", cudaGetErrorString(e));
  return DZS_OK;
}

// per-stage event pair on the context stream (no synchronisation)
cudaEvent_t prof_event(dzs_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

struct ProfScope {
  dzs_ctx* c;
  int cat;
  cudaEvent_t a = nullptr;
  ProfScope(dzs_ctx* cc, int k) : c(cc), cat(k) {
    if (c->prof_on) {
      a = prof_event(c);
      cudaEventRecord(a, c->stream);
    }
  }
  ~ProfScope() {
    if (c->prof_on && a) {
      cudaEvent_t b = prof_event(c);
      cudaEventRecord(b, c->stream);
      c->prof_pending.push_back({cat, a, b});
    }
  }
};

// forces of the current (sorted) particle set: tree, PM, walk (+ closing kick)
void run_force(dzs_ctx* c, int parts, bool close_kick) {
  {
    ProfScope ps(c, DZS_PROF_TREE);
    launch_tree(c);  // also lists the groups the walk needs
  }
  if (parts & DZS_ACC_PM) {
    {
      ProfScope ps(c, DZS_PROF_PM);
      launch_pm_deposit(c);
    }
    {
      ProfScope ps(c, DZS_PROF_FFT);
      launch_pm_fft(c);
    }
    ProfScope ps(c, DZS_PROF_PM);
    launch_pm_interp(c);
  } else {
    cudaMemsetAsync(c->B.g, 0, 3 * c->cap * (c->fp64 ? 8 : 4), c->stream);
  }
  ProfScope ps(c, DZS_PROF_WALK);
  launch_walk(c, (parts & DZS_ACC_TREE) != 0, close_kick, c->step);
}

// forces of the current state in its current order (sorts a copy of the
// order, computes, restores the order); g in double, stride n, in convert
void force_in_order(dzs_ctx* c, int parts) {
  launch_keys(c);
  launch_sort(c);
  run_force(c, parts, false);
  launch_unpermute(c, (double*)c->B.convert);
}

}  // namespace

extern "C" {

dzs_status dzs_params_default(dzs_params* p) {
  if (!p) return DZS_EINVAL;
  memset(p, 0, sizeof(*p));
  p->n1d = 32;
  p->mesh = 64;
  p->box = 64.0;
  p->omega_m = 0.3;
  p->omega_l = 0.7;
  p->hubble = 0.7;
  p->sigma8 = 0.8;
  p->ns = 0.96;
  p->z_init = 49.0;
  p->nsteps = 96;
  p->leaf_bucket = 8;
  p->walk_group = 32;
  p->dzs_on = 1;
  p->merge_level = 2;
  p->rlc_mode = DZS_RLC_SWEEP;
  p->rs_cells = 1.25;
  p->rcut_rs = 4.5;
  p->theta = 0.5;
  p->soft_frac = 1.0 / 40.0;
  p->theta_dzs = 0.1;
  p->buffer_cells = 2.0;
  p->seed = 1;
  p->precision = DZS_FP32;
  p->device = 0;
  p->lc_capacity = 0;
  p->dzs_criterion = DZS_CRIT_GEOMETRIC;
  p->alpha_dyn = 0.01;
  return DZS_OK;
}

dzs_status dzs_footprint_bytes(const dzs_params* p, size_t* bytes) {
  const char* why = validate(p);
  if (why || !bytes) return fail(nullptr, DZS_EINVAL, why ? why : "bytes is NULL");
  *bytes = Plan(*p).total;
  return DZS_OK;
}

dzs_status dzs_create(const dzs_params* p, void* cuda_stream, dzs_ctx** out) {
  if (!out) return fail(nullptr, DZS_EINVAL, "out is NULL");
  *out = nullptr;
  const char* why = validate(p);
  if (why) return fail(nullptr, DZS_EINVAL, why);
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || p->device < 0 || p->device >= ndev)
    return fail(nullptr, DZS_EDEVICE, "no such CUDA device");
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, p->device) != cudaSuccess) return fail(nullptr, DZS_EDEVICE, "device query");
  if (!(prop.major == 10 && prop.minor == 3))
    return fail(nullptr, DZS_EDEVICE, "this library is built for sm_103a (GB300) only");
  dzs_ctx* c = new (std::nothrow) dzs_ctx();
  if (!c) return fail(nullptr, DZS_ENOMEM, "host allocation");
  c->P = *p;
  c->dev = p->device;
  c->stream = (cudaStream_t)cuda_stream;
  c->fp64 = p->precision == DZS_FP64;
  c->n1 = p->n1d;
  c->N0 = (int64_t)p->n1d * p->n1d * p->n1d;
  c->cap = p->capacity ? (int64_t)p->capacity : c->N0;
  c->M = p->mesh;
  c->mesh_pow2 = is_pow2(p->mesh);
  c->logM = ilog2i(p->mesh) - (c->mesh_pow2 ? 0 : 1);  // floor(log2 M): depth of the Morton cell table
  c->lat = 4294967296.0 / p->box;
  c->scale = p->box / 4294967296.0;
  c->gm0 = 1.5 * p->omega_m * p->box * p->box * p->box / (4.0 * M_PI * (double)c->N0);
  c->eps0 = p->soft_frac * p->box / p->n1d;
  c->rs = p->rs_cells * p->box / p->mesh;
  c->rcut = p->rcut_rs * c->rs;
  {
    // same operation order as the definition r_cut / L * 2^32
    double rcut_lat = p->rcut_rs * c->rs / p->box * 4294967296.0;
    c->rcut_lat2 = rcut_lat * rcut_lat;
  }
  // the walk keeps a node when (double)gap2 <= r_cut_lat^2 and opens it when
  // (double)l >= theta * sqrt((double)dcom2); both are monotone in the integer
  // squared distance, so each becomes "d2 <= largest d2 that passes"
  c->walk_skip_d2 = largest_passing([&](uint64_t x) { return (double)x <= c->rcut_lat2; });
  for (int l = 0; l <= kMaxLevel; ++l) {
    double side = std::ldexp(1.0, 32 - l);
    double th = p->theta;
    c->walk_open_d2[l] = largest_passing([&](uint64_t x) { return side >= th * std::sqrt((double)x); });
  }
  int j = 1;
  while (((int64_t)1 << j) * ((int64_t)1 << (p->merge_level - 1)) < p->n1d) ++j;
  c->jmin = j;
  c->blat = (uint64_t)std::floor(p->buffer_cells * 4294967296.0 / p->mesh);
  for (int l = 0; l <= kMaxLevel; ++l) {
    double lovt = std::ceil(std::ldexp(1.0, 32 - l) / p->theta_dzs);
    c->merge_thr[l] = (lovt < 4294967296.0) ? c->blat + (uint64_t)lovt : ~0ull;
  }
  compute_tables(c->P, c->T);
  Plan pl(*p);
  c->node_cap = pl.node_cap;
  c->ring_cap = (size_t)pl.ring;
  dzs_status st = DZS_OK;
  if (cudaSetDevice(c->dev) != cudaSuccess) {
    delete c;
    return fail(nullptr, DZS_EDEVICE, "cudaSetDevice");
  }
  cudaError_t e = dev_alloc((void**)&c->arena, pl.total);
  if (e != cudaSuccess) {
    delete c;
    return fail(nullptr, DZS_ENOMEM, "device arena", cudaGetErrorString(e));
  }
  c->arena_bytes = pl.total;
  char* a = c->arena;
  Buffers& B = c->B;
  B.u = (uint32_t*)(a + pl.o_u);
  B.u2 = (uint32_t*)(a + pl.o_u2);
  B.p = a + pl.o_p;
  B.p2 = a + pl.o_p2;
  B.g = a + pl.o_g;
  B.gsave = a + pl.o_gsave;
  B.k = (uint32_t*)(a + pl.o_k);
  B.k2 = (uint32_t*)(a + pl.o_k2);
  B.id = (uint32_t*)(a + pl.o_id);
  B.id2 = (uint32_t*)(a + pl.o_id2);
  B.fl = (uint8_t*)(a + pl.o_fl);
  B.fl2 = (uint8_t*)(a + pl.o_fl2);
  B.key = (uint64_t*)(a + pl.o_key);
  B.key2 = (uint64_t*)(a + pl.o_key2);
  B.idx = (uint32_t*)(a + pl.o_idx);
  B.idx2 = (uint32_t*)(a + pl.o_idx2);
  B.hist = (uint32_t*)(a + pl.o_hist);
  B.blocksum = (int64_t*)(a + pl.o_blocksum);
  B.iscan = (int32_t*)(a + pl.o_iscan);
  B.prefix = (uint64_t*)(a + pl.o_prefix);
  B.mend = (int32_t*)(a + pl.o_mend);
  B.nodes = (Node*)(a + pl.o_nodes);
  B.lvl_count = (int32_t*)(a + pl.o_lvl);
  B.cfirst = (int32_t*)(a + pl.o_cfirst);
  B.parent = (int32_t*)(a + pl.o_parent);
  B.cicw = a + pl.o_cicw;
  B.groups = (int32_t*)(a + pl.o_groups);
  B.group_head = (int32_t*)(a + pl.o_ghead);
  B.wpm = a + pl.o_wpm;
  B.wph = a + pl.o_wph;
  B.wnh = a + pl.o_wnh;
  B.wlen = (int32_t*)(a + pl.o_wlen);
  B.rho = a + pl.o_rho;
  B.spec = a + pl.o_spec;
  B.phi = a + pl.o_phi;
  B.cell_start = (int32_t*)(a + pl.o_cstart);
  B.twiddle = a + pl.o_tw;
  B.green_axis = a + pl.o_green;
  B.ring = (dzs_lc_record*)(a + pl.o_ring);
  B.n = (int32_t*)(a + pl.o_n);
  B.err = (uint32_t*)(a + pl.o_err);
  B.counters = (uint64_t*)(a + pl.o_counters);
  B.diag = (double*)(a + pl.o_diag);
  B.convert = a + pl.o_convert;
  if (cudaMemset(B.n, 0, 16) != cudaSuccess || cudaMemset(B.err, 0, 16) != cudaSuccess ||
      cudaMemset(B.counters, 0, 8 * 32) != cudaSuccess) {
    cudaFree(c->arena);
    delete c;
    return fail(nullptr, DZS_ECUDA, "arena init");
  }
  launch_fft_init(c);
  if (cudaDeviceSynchronize() != cudaSuccess) st = DZS_ECUDA;
  if (st != DZS_OK) {
    cudaFree(c->arena);
    delete c;
    return fail(nullptr, st, "context init");
  }
  *out = c;
  return DZS_OK;
}

dzs_status dzs_destroy(dzs_ctx* c) {
  if (!c) return DZS_OK;
  cudaSetDevice(c->dev);
  cudaStreamSynchronize(c->stream);
  for (auto& pe : c->prof_pending) {
    cudaEventDestroy(pe.a);
    cudaEventDestroy(pe.b);
  }
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  for (cudaEvent_t e : c->pipe_ev)
    if (e) cudaEventDestroy(e);
  if (c->pipe) cudaFreeHost(c->pipe);
  if (c->copy_stream) {
    cudaStreamSynchronize(c->copy_stream);
    cudaStreamDestroy(c->copy_stream);
  }
  if (c->arena) cudaFree(c->arena);
  if (c->obs.sky) cudaFree(c->obs.sky);
  if (c->obs.grid) cudaFree(c->obs.grid);
  if (c->sht_work) cudaFree(c->sht_work);
  delete c;
  return DZS_OK;
}

dzs_status dzs_ics(dzs_ctx* c) {
  dzs_status s = guard(c);
  if (s) return s;
  if (c->cap != c->N0) return fail(c, DZS_EINVAL, "dzs_ics needs capacity n1d^3");
  CK(cudaMemsetAsync(c->B.counters, 0, 8 * 32, c->stream));
  CK(cudaMemsetAsync(c->B.err, 0, 16, c->stream));
  c->drained = 0;
  launch_ics(c);
  c->step = 0;
  launch_keys(c);
  launch_sort(c);
  run_force(c, DZS_ACC_ALL, false);
  c->have_state = true;
  c->g_aligned = true;
  c->amin2_ready = false;
  CK(cudaGetLastError());
  return check_device_errors(c);
}

dzs_status dzs_run_stages(dzs_ctx* c, uint32_t mask) {
  dzs_status s = guard(c);
  if (s) return s;
  if (!c->have_state) return fail(c, DZS_ESTATE, "no particle state (call dzs_ics or dzs_set_state)");
  if (c->step >= c->P.nsteps && (mask & (DZS_STAGE_KICK_DRIFT | DZS_STAGE_CLOSE | DZS_STAGE_MERGE)))
    return fail(c, DZS_ESTATE, "the run has reached a = 1");
  const int st = c->step;
  if (mask & DZS_STAGE_KICK_DRIFT) {
    ProfScope ps(c, DZS_PROF_KICK_DRIFT);
    launch_kick_drift(c, st, true, true);
    launch_records(c, st);
    // a_min of the dynamical criterion: the accelerations the particles were
    // just kicked with, restricted to those not crossed after this drift
    if (c->P.dzs_on && c->P.dzs_criterion == DZS_CRIT_DYNAMICAL) launch_amin2(c);
  }
  if (mask & DZS_STAGE_SORT) {
    ProfScope ps(c, DZS_PROF_SORT);
    if (!(mask & DZS_STAGE_KICK_DRIFT)) launch_keys(c);
    launch_sort(c);
    c->g_aligned = false;  // the sort permutes the state but not g
  }
  if ((mask & DZS_STAGE_MERGE) && c->P.dzs_on) {
    ProfScope ps(c, DZS_PROF_MERGE);
    if (c->P.dzs_criterion == DZS_CRIT_DYNAMICAL && !c->amin2_ready) {
      if (!c->g_aligned)
        return fail(c, DZS_ESTATE, "dynamical criterion: a_min needs the kick-drift stage before the sort");
      launch_amin2(c);
    }
    launch_merge(c, c->T.rlat[st + 1]);
    c->g_aligned = false;  // the merge compacts the state but not g
  }
  if (mask & DZS_STAGE_FORCE) {
    run_force(c, DZS_ACC_ALL, (mask & DZS_STAGE_CLOSE) != 0);
    c->g_aligned = true;
  } else if (mask & DZS_STAGE_CLOSE) {
    ProfScope ps(c, DZS_PROF_WALK);
    launch_close_kick(c, st);
  }
  if (mask & DZS_STAGE_CLOSE) {
    c->step = st + 1;
    c->amin2_ready = false;
  }
  CK(cudaGetLastError());
  return DZS_OK;
}

// Before a full step: a ring smaller than N0 may not hold the step's records
// (with ring_cap >= N0 it always does: the records pending plus those still to
// come are distinct particles, each recorded once).  A dry run of the step's
// kick, drift and crossing test counts them (synchronises); if they do not
// fit, the step is not started and the caller drains and steps again.
dzs_status ring_guard(dzs_ctx* c) {
  if (c->ring_cap >= (size_t)c->N0 || c->step >= c->P.nsteps) return DZS_OK;
  unsigned long long* cnt = (unsigned long long*)(c->B.counters + 18);
  CK(cudaMemsetAsync(cnt, 0, sizeof(uint64_t), c->stream));
  launch_count_crossings(c, c->step, cnt);
  uint64_t ctr[19];
  CK(cudaMemcpyAsync(ctr, c->B.counters, sizeof ctr, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const uint64_t pending = ctr[0] - c->drained;
  const uint64_t room = c->ring_cap > pending ? c->ring_cap - pending : 0;
  if (ctr[18] > room) {
    char buf[160];
    snprintf(buf, sizeof buf, "lightcone ring full: step %d would record %llu, room %llu; drain and step again",
             (int)c->step, (unsigned long long)ctr[18], (unsigned long long)room);
    return fail(c, DZS_EOVERFLOW, buf);
  }
  return DZS_OK;
}

// end of a step in pipelined mode: its diagnostics, ring counters and error
// word copied to the step's pinned slot behind the step's kernels; the slot of
// the step kPipe earlier is reused once its copies have landed
dzs_status pipe_record(dzs_ctx* c) {
  const int32_t s = c->step;
  const int k = s % dzs_ctx::kPipe;
  CK(cudaEventSynchronize(c->pipe_ev[k]));
  launch_diagnostics(c);
  dzs_ctx::PipeSlot* slot = c->pipe + k;
  CK(cudaMemcpyAsync(slot->diag, c->B.diag, sizeof slot->diag, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(slot->ring, c->B.counters, sizeof slot->ring, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(slot->err, c->B.err, sizeof slot->err, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaEventRecord(c->pipe_ev[k], c->stream));
  c->pipe_step[k] = s;
  return DZS_OK;
}

dzs_status dzs_step(dzs_ctx* c, int32_t nsteps, int32_t* steps_done) {
  dzs_status s = guard(c);
  if (s) return s;
  if (steps_done) *steps_done = 0;
  if (nsteps < 0) return fail(c, DZS_EINVAL, "nsteps < 0");
  int done = 0;
  while (done < nsteps && c->step < c->P.nsteps) {
    s = ring_guard(c);
    if (!s) s = dzs_run_stages(c, DZS_STAGE_ALL);
    if (!s && c->pipe_on) s = pipe_record(c);
    if (s) {
      if (steps_done) *steps_done = done;
      return s;
    }
    ++done;
  }
  if (steps_done) *steps_done = done;
  return DZS_OK;
}

dzs_status dzs_step_until(dzs_ctx* c, int32_t max_steps, const dzs_halt* h, int32_t* steps_done,
                          int32_t* reason, double* ratio) {
  dzs_status s = guard(c);
  if (s) return s;
  if (steps_done) *steps_done = 0;
  if (reason) *reason = DZS_HALT_NONE;
  if (max_steps < 0 || !h || !(h->ratio_min >= 0) || !(h->wall_limit_s >= 0) || !(h->horizon_s >= 0))
    return fail(c, DZS_EINVAL, "bad halt arguments");
  if (!c->have_state) return fail(c, DZS_ESTATE, "no particle state");
  using clk = std::chrono::steady_clock;
  const clk::time_point t0 = clk::now();
  size_t n = 0;
  s = dzs_get_count(c, &n, nullptr);
  if (s) return s;
  double r0 = (double)n / (double)c->N0, r = r0;
  if (ratio) *ratio = r;
  int done = 0;
  while (done < max_steps && c->step < c->P.nsteps) {
    s = ring_guard(c);
    if (!s) s = dzs_run_stages(c, DZS_STAGE_ALL);
    if (s) return s;
    ++done;
    if (steps_done) *steps_done = done;
    s = dzs_get_count(c, &n, nullptr);  // synchronises
    if (s) return s;
    r = (double)n / (double)c->N0;
    if (ratio) *ratio = r;
    if (h->ratio_min > 0 && r < h->ratio_min) {
      if (reason) *reason = DZS_HALT_RATIO;
      return DZS_OK;
    }
    const double t = std::chrono::duration<double>(clk::now() - t0).count();
    if (h->wall_limit_s > 0 && t >= h->wall_limit_s) {
      // linear extrapolation of R(t) over this call's steps
      const double slope = (r - r0) / t;
      const bool soon = h->ratio_min > 0 && r + slope * h->horizon_s < h->ratio_min;
      if (reason) *reason = soon ? DZS_HALT_PREDICTED : DZS_HALT_WALL;
      return DZS_OK;
    }
  }
  return DZS_OK;
}

dzs_status dzs_lightcone_drain(dzs_ctx* c, dzs_lc_record* host_buf, size_t cap, size_t* n_out) {
  dzs_status s = guard(c);
  if (s) return s;
  if (n_out) *n_out = 0;
  if (!host_buf && cap) return fail(c, DZS_EINVAL, "host_buf is NULL");
  s = check_device_errors(c);
  if (s) return s;
  uint64_t ctr[2];
  CK(cudaMemcpy(ctr, c->B.counters, sizeof ctr, cudaMemcpyDeviceToHost));
  uint64_t avail = ctr[0] - c->drained;
  uint64_t take = avail < cap ? avail : cap;
  uint64_t done = 0;
  while (done < take) {
    uint64_t slot = (c->drained + done) % c->ring_cap;
    uint64_t chunk = c->ring_cap - slot;
    if (chunk > take - done) chunk = take - done;
    CK(cudaMemcpy(host_buf + done, c->B.ring + slot, chunk * sizeof(dzs_lc_record), cudaMemcpyDeviceToHost));
    done += chunk;
  }
  c->drained += take;
  if (n_out) *n_out = (size_t)take;
  if (ctr[1]) {
    char buf[128];
    snprintf(buf, sizeof buf, "%llu lightcone records dropped (ring full)", (unsigned long long)ctr[1]);
    return fail(c, DZS_EOVERFLOW, buf);
  }
  return DZS_OK;
}

dzs_status dzs_pipeline(dzs_ctx* c, int32_t on) {
  dzs_status s = guard(c);
  if (s) return s;
  if (on && !c->pipe) {
    CK(cudaHostAlloc((void**)&c->pipe, sizeof(dzs_ctx::PipeSlot) * dzs_ctx::kPipe, cudaHostAllocDefault));
    for (int k = 0; k < dzs_ctx::kPipe; ++k) CK(cudaEventCreateWithFlags(&c->pipe_ev[k], cudaEventDisableTiming));
    CK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
  }
  if (!on) CK(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < dzs_ctx::kPipe; ++k) c->pipe_step[k] = -1;
  c->pipe_on = on != 0;
  return DZS_OK;
}

namespace {
// the pinned slot holding completed-step count `step`, after its copies landed
dzs_status pipe_slot(dzs_ctx* c, int32_t step, const dzs_ctx::PipeSlot** out) {
  if (!c->pipe_on) return fail(c, DZS_ESTATE, "pipelined results are off (dzs_pipeline)");
  const int k = ((step % dzs_ctx::kPipe) + dzs_ctx::kPipe) % dzs_ctx::kPipe;
  if (step < 0 || c->pipe_step[k] != step)
    return fail(c, DZS_EINVAL, "no result kept for that step (only the last 4 steps are)");
  CK(cudaEventSynchronize(c->pipe_ev[k]));
  const dzs_ctx::PipeSlot* slot = c->pipe + k;
  if (slot->err[0] & (kErrNodes | kErrStack | kErrGroups)) {
    char buf[160];
    snprintf(buf, sizeof buf, "device buffer overflow (error word 0x%x)", slot->err[0]);
    return fail(c, DZS_EOVERFLOW, buf);
  }
  *out = slot;
  return DZS_OK;
}
}  // namespace

dzs_status dzs_step_result(dzs_ctx* c, int32_t step, double diag[8], uint64_t* lc_written) {
  dzs_status s = guard(c);
  if (s) return s;
  const dzs_ctx::PipeSlot* slot = nullptr;
  s = pipe_slot(c, step, &slot);
  if (s) return s;
  if (diag) std::memcpy(diag, slot->diag, sizeof slot->diag);
  if (lc_written) *lc_written = slot->ring[0];
  return DZS_OK;
}

dzs_status dzs_lightcone_drain_step(dzs_ctx* c, int32_t step, dzs_lc_record* host_buf, size_t cap, size_t* n_out) {
  dzs_status s = guard(c);
  if (s) return s;
  if (n_out) *n_out = 0;
  if (!host_buf && cap) return fail(c, DZS_EINVAL, "host_buf is NULL");
  const dzs_ctx::PipeSlot* slot = nullptr;
  s = pipe_slot(c, step, &slot);
  if (s) return s;
  // records [drained, head of that step) are complete and stay in place while
  // later steps append: copied on the copy stream beside the running kernels
  const uint64_t head = slot->ring[0];
  const uint64_t avail = head > c->drained ? head - c->drained : 0;
  const uint64_t take = avail < cap ? avail : cap;
  uint64_t done = 0;
  while (done < take) {
    const uint64_t ring_slot = (c->drained + done) % c->ring_cap;
    uint64_t chunk = c->ring_cap - ring_slot;
    if (chunk > take - done) chunk = take - done;
    CK(cudaMemcpyAsync(host_buf + done, c->B.ring + ring_slot, chunk * sizeof(dzs_lc_record), cudaMemcpyDeviceToHost,
                       c->copy_stream));
    done += chunk;
  }
  CK(cudaStreamSynchronize(c->copy_stream));
  c->drained += take;
  if (n_out) *n_out = (size_t)take;
  if (slot->ring[1]) {
    char buf[128];
    snprintf(buf, sizeof buf, "%llu lightcone records dropped (ring full)", (unsigned long long)slot->ring[1]);
    return fail(c, DZS_EOVERFLOW, buf);
  }
  return DZS_OK;
}

dzs_status dzs_get_count(dzs_ctx* c, size_t* n, int32_t* step) {
  dzs_status s = guard(c);
  if (s) return s;
  s = check_device_errors(c);
  if (s) return s;
  int32_t hn = 0;
  CK(cudaMemcpy(&hn, c->B.n, sizeof hn, cudaMemcpyDeviceToHost));
  if (n) *n = (size_t)hn;
  if (step) *step = c->step;
  return DZS_OK;
}

dzs_status dzs_get_state(dzs_ctx* c, uint32_t* u, double* p, double* g, uint32_t* k, uint32_t* id, uint8_t* fl,
                         size_t cap, size_t* n_out) {
  size_t n = 0;
  dzs_status s = dzs_get_count(c, &n, nullptr);
  if (s) return s;
  if (n_out) *n_out = n;
  if (n > cap) return fail(c, DZS_EINVAL, "cap smaller than the particle count");
  double* conv = (double*)c->B.convert;
  for (int ax = 0; ax < 3; ++ax) {
    if (u) CK(cudaMemcpy(u + ax * n, c->B.u + ax * c->cap, 4 * n, cudaMemcpyDeviceToHost));
  }
  if (p) {
    launch_to_double(c, c->B.p, 3 * c->cap, conv);
    CK(cudaStreamSynchronize(c->stream));
    for (int ax = 0; ax < 3; ++ax)
      CK(cudaMemcpy(p + ax * n, conv + ax * c->cap, 8 * n, cudaMemcpyDeviceToHost));
  }
  if (g) {
    launch_to_double(c, c->B.g, 3 * c->cap, conv);
    CK(cudaStreamSynchronize(c->stream));
    for (int ax = 0; ax < 3; ++ax)
      CK(cudaMemcpy(g + ax * n, conv + ax * c->cap, 8 * n, cudaMemcpyDeviceToHost));
  }
  if (k) CK(cudaMemcpy(k, c->B.k, 4 * n, cudaMemcpyDeviceToHost));
  if (id) CK(cudaMemcpy(id, c->B.id, 4 * n, cudaMemcpyDeviceToHost));
  if (fl) {
    CK(cudaMemcpy(fl, c->B.fl, n, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < n; ++i) fl[i] &= (uint8_t)(DZS_FL_CROSSED | DZS_FL_MERGED);
  }
  return DZS_OK;
}

dzs_status dzs_set_state(dzs_ctx* c, const uint32_t* u, const double* p, const double* g, const uint32_t* k,
                         const uint32_t* id, const uint8_t* fl, size_t n, int32_t step) {
  dzs_status s = guard(c);
  if (s) return s;
  if (n > (size_t)c->cap) return fail(c, DZS_EINVAL, "n exceeds the context's capacity");
  if (n > 0 && (!u || !p || !k || !id || !fl)) return fail(c, DZS_EINVAL, "NULL state array");
  if (step < 0 || step > c->P.nsteps) return fail(c, DZS_EINVAL, "step out of range");
  CK(cudaStreamSynchronize(c->stream));
  double* conv = (double*)c->B.convert;
  for (int ax = 0; ax < 3; ++ax) {
    CK(cudaMemcpy(c->B.u + ax * c->cap, u + ax * n, 4 * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(conv + ax * c->cap, p + ax * n, 8 * n, cudaMemcpyHostToDevice));
  }
  launch_from_double(c, conv, 3 * c->cap, c->B.p);
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(c->B.k, k, 4 * n, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->B.id, id, 4 * n, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->B.fl, fl, n, cudaMemcpyHostToDevice));
  int32_t nn = (int32_t)n;
  CK(cudaMemcpy(c->B.n, &nn, sizeof nn, cudaMemcpyHostToDevice));
  CK(cudaMemset(c->B.err, 0, 16));
  CK(cudaMemset(c->B.counters + 4, 0, 4 * sizeof(uint64_t)));  // pairs and stack depth (4, 7)
  CK(cudaMemset(c->B.counters + 12, 0, 2 * sizeof(uint64_t)));  // node tests, rounds
  CK(cudaMemset(c->B.counters + 20, 0, 2 * sizeof(uint64_t)));  // window starts, fallbacks
  c->step = step;
  c->have_state = true;
  c->g_aligned = true;
  c->amin2_ready = false;
  if (g) {
    for (int ax = 0; ax < 3; ++ax)
      CK(cudaMemcpy(conv + ax * c->cap, g + ax * n, 8 * n, cudaMemcpyHostToDevice));
    launch_from_double(c, conv, 3 * c->cap, c->B.g);
  } else {
    force_in_order(c, DZS_ACC_ALL);  // g (double, stride n) in convert
    size_t rs = c->fp64 ? 8 : 4;
    for (int ax = 0; ax < 3; ++ax)
      launch_from_double(c, conv + ax * n, (int64_t)n, (char*)c->B.g + ax * c->cap * rs);
  }
  CK(cudaGetLastError());
  return check_device_errors(c);
}

dzs_status dzs_accel(dzs_ctx* c, int32_t parts, double* g_out) {
  dzs_status s = guard(c);
  if (s) return s;
  if (!g_out || parts < 1 || parts > 3) return fail(c, DZS_EINVAL, "bad arguments");
  if (!c->have_state) return fail(c, DZS_ESTATE, "no particle state");
  size_t n = 0;
  s = dzs_get_count(c, &n, nullptr);
  if (s) return s;
  // keep the state's g: force_in_order overwrites it
  double* conv = (double*)c->B.convert;
  size_t gbytes = 3 * c->cap * (c->fp64 ? 8 : 4);
  CK(cudaMemcpyAsync(c->B.gsave, c->B.g, gbytes, cudaMemcpyDeviceToDevice, c->stream));
  force_in_order(c, parts);
  CK(cudaMemcpyAsync(c->B.g, c->B.gsave, gbytes, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaGetLastError());
  s = check_device_errors(c);
  if (s) return s;
  CK(cudaMemcpy(g_out, conv, 8 * 3 * n, cudaMemcpyDeviceToHost));
  return DZS_OK;
}

dzs_status dzs_merge_only(dzs_ctx* c, uint64_t rlat) {
  dzs_status s = guard(c);
  if (s) return s;
  if (!c->have_state) return fail(c, DZS_ESTATE, "no particle state");
  if (c->P.dzs_criterion == DZS_CRIT_DYNAMICAL) {
    if (!c->g_aligned) return fail(c, DZS_ESTATE, "dynamical criterion: g is not in the state's order");
    launch_amin2(c);
  }
  launch_keys(c);
  launch_merge(c, rlat);
  c->g_aligned = false;
  CK(cudaGetLastError());
  return check_device_errors(c);
}

dzs_status dzs_diagnostics(dzs_ctx* c, double out[8]) {
  dzs_status s = guard(c);
  if (s) return s;
  if (!out) return fail(c, DZS_EINVAL, "out is NULL");
  launch_diagnostics(c);
  CK(cudaGetLastError());
  s = check_device_errors(c);
  if (s) return s;
  CK(cudaMemcpy(out, c->B.diag, 8 * sizeof(double), cudaMemcpyDeviceToHost));
  return DZS_OK;
}

// ---- checkpoint / restore: header, raw state arrays in the context's own
// precision (no conversion, so a restored run continues bit for bit), and the
// lightcone records not yet drained
namespace {
constexpr uint64_t kCkptMagic = 0x315450434b535a44ull;  // "DZSKCPT1"
struct CkptHeader {
  uint64_t magic;
  uint64_t bytes;
  dzs_params params;
  uint64_t n, step, pending, dropped, rsz;
};
size_t ckpt_size(const dzs_ctx* c, uint64_t n, uint64_t pending) {
  size_t rsz = c->fp64 ? 8 : 4;
  return sizeof(CkptHeader) + n * (12 + 6 * rsz + 4 + 4 + 1) + pending * sizeof(dzs_lc_record);
}
bool same_physics(const dzs_params& a, const dzs_params& b) {
  dzs_params x = a, y = b;
  x.device = y.device = 0;
  x.lc_capacity = y.lc_capacity = 0;
  x.capacity = y.capacity = 0;
  x.walk_eval = y.walk_eval = 0;  // execution only
  return memcmp(&x, &y, sizeof x) == 0;
}
}  // namespace

dzs_status dzs_checkpoint_bytes(dzs_ctx* c, size_t* bytes) {
  size_t n = 0;
  dzs_status s = dzs_get_count(c, &n, nullptr);
  if (s) return s;
  if (!bytes) return fail(c, DZS_EINVAL, "bytes is NULL");
  uint64_t head = 0;
  CK(cudaMemcpy(&head, c->B.counters, sizeof head, cudaMemcpyDeviceToHost));
  *bytes = ckpt_size(c, n, head - c->drained);
  return DZS_OK;
}

dzs_status dzs_checkpoint(dzs_ctx* c, void* host_buf, size_t cap, size_t* written) {
  size_t n = 0;
  dzs_status s = dzs_get_count(c, &n, nullptr);
  if (s) return s;
  if (!c->have_state) return fail(c, DZS_ESTATE, "no particle state");
  uint64_t ctr[2];
  CK(cudaMemcpy(ctr, c->B.counters, sizeof ctr, cudaMemcpyDeviceToHost));
  const uint64_t pending = ctr[0] - c->drained;
  const size_t need = ckpt_size(c, n, pending), rsz = c->fp64 ? 8 : 4;
  if (written) *written = 0;
  if (!host_buf || cap < need) return fail(c, DZS_EINVAL, "checkpoint buffer too small");
  char* o = (char*)host_buf;
  CkptHeader h;
  memset(&h, 0, sizeof h);
  h.magic = kCkptMagic;
  h.bytes = need;
  h.params = c->P;
  h.n = n;
  h.step = (uint64_t)c->step;
  h.pending = pending;
  h.dropped = ctr[1];
  h.rsz = rsz;
  memcpy(o, &h, sizeof h);
  o += sizeof h;
  for (int ax = 0; ax < 3; ++ax, o += 4 * n) CK(cudaMemcpy(o, c->B.u + ax * c->cap, 4 * n, cudaMemcpyDeviceToHost));
  for (int ax = 0; ax < 3; ++ax, o += rsz * n)
    CK(cudaMemcpy(o, (char*)c->B.p + ax * c->cap * rsz, rsz * n, cudaMemcpyDeviceToHost));
  for (int ax = 0; ax < 3; ++ax, o += rsz * n)
    CK(cudaMemcpy(o, (char*)c->B.g + ax * c->cap * rsz, rsz * n, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(o, c->B.k, 4 * n, cudaMemcpyDeviceToHost));
  o += 4 * n;
  CK(cudaMemcpy(o, c->B.id, 4 * n, cudaMemcpyDeviceToHost));
  o += 4 * n;
  CK(cudaMemcpy(o, c->B.fl, n, cudaMemcpyDeviceToHost));
  o += n;
  for (uint64_t done = 0; done < pending;) {
    uint64_t slot = (c->drained + done) % c->ring_cap, chunk = c->ring_cap - slot;
    if (chunk > pending - done) chunk = pending - done;
    CK(cudaMemcpy(o, c->B.ring + slot, chunk * sizeof(dzs_lc_record), cudaMemcpyDeviceToHost));
    o += chunk * sizeof(dzs_lc_record);
    done += chunk;
  }
  if (written) *written = need;
  return DZS_OK;
}

dzs_status dzs_restore(dzs_ctx* c, const void* host_buf, size_t len) {
  dzs_status s = guard(c);
  if (s) return s;
  CkptHeader h;
  if (!host_buf || len < sizeof h) return fail(c, DZS_EINVAL, "checkpoint too short");
  memcpy(&h, host_buf, sizeof h);
  const size_t rsz = c->fp64 ? 8 : 4;
  if (h.magic != kCkptMagic || h.rsz != rsz) return fail(c, DZS_EINVAL, "not a checkpoint of this precision");
  if (!same_physics(h.params, c->P)) return fail(c, DZS_EINVAL, "checkpoint parameters differ from the context's");
  if (h.n > (uint64_t)c->cap || h.step > (uint64_t)c->P.nsteps || h.pending > c->ring_cap ||
      h.bytes != ckpt_size(c, h.n, h.pending) || len < h.bytes)
    return fail(c, DZS_EINVAL, "inconsistent checkpoint");
  CK(cudaStreamSynchronize(c->stream));
  const size_t n = h.n;
  const char* o = (const char*)host_buf + sizeof h;
  for (int ax = 0; ax < 3; ++ax, o += 4 * n) CK(cudaMemcpy(c->B.u + ax * c->cap, o, 4 * n, cudaMemcpyHostToDevice));
  for (int ax = 0; ax < 3; ++ax, o += rsz * n)
    CK(cudaMemcpy((char*)c->B.p + ax * c->cap * rsz, o, rsz * n, cudaMemcpyHostToDevice));
  for (int ax = 0; ax < 3; ++ax, o += rsz * n)
    CK(cudaMemcpy((char*)c->B.g + ax * c->cap * rsz, o, rsz * n, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->B.k, o, 4 * n, cudaMemcpyHostToDevice));
  o += 4 * n;
  CK(cudaMemcpy(c->B.id, o, 4 * n, cudaMemcpyHostToDevice));
  o += 4 * n;
  CK(cudaMemcpy(c->B.fl, o, n, cudaMemcpyHostToDevice));
  o += n;
  if (h.pending) CK(cudaMemcpy(c->B.ring, o, h.pending * sizeof(dzs_lc_record), cudaMemcpyHostToDevice));
  uint64_t ctr[2] = {h.pending, h.dropped};
  CK(cudaMemcpy(c->B.counters, ctr, sizeof ctr, cudaMemcpyHostToDevice));
  int32_t nn = (int32_t)n;
  CK(cudaMemcpy(c->B.n, &nn, sizeof nn, cudaMemcpyHostToDevice));
  CK(cudaMemset(c->B.err, 0, 16));
  c->drained = 0;
  c->step = (int32_t)h.step;
  c->have_state = true;
  c->g_aligned = true;
  c->amin2_ready = false;
  return DZS_OK;
}

// ---- lightcone observables
dzs_status dzs_observe_enable(dzs_ctx* c, const dzs_observe* o) {
  dzs_status s = guard(c);
  if (s) return s;
  const bool off = !o || (o->nside == 0 && o->mesh == 0);
  if (!off) {
    const bool pow2 = o->nside > 0 && (o->nside & (o->nside - 1)) == 0;
    if (o->nside < 0 || (o->nside != 0 && (!pow2 || o->nside > 4096)) || o->mesh < 0 || o->mesh > 1024 ||
        !(o->a_lo <= o->a_hi))
      return fail(c, DZS_EINVAL, "bad observables (nside a power of two <= 4096, mesh <= 1024, a_lo <= a_hi)");
  }
  CK(cudaStreamSynchronize(c->stream));
  if (c->obs.sky) CK(cudaFree(c->obs.sky));
  if (c->obs.grid) CK(cudaFree(c->obs.grid));
  c->obs = dzs::ObserveTarget();
  if (off) return DZS_OK;
  dzs::ObserveTarget t;
  t.nside = o->nside;
  t.mesh = o->mesh;
  t.a_lo = o->a_lo;
  t.a_hi = o->a_hi;
  t.half = 0.5 * c->P.box;
  t.box = c->P.box;
  if (t.nside) {
    const size_t b = 8 * (size_t)(12 * t.nside * t.nside);
    if (dev_alloc((void**)&t.sky, b) != cudaSuccess) return fail(c, DZS_ENOMEM, "sky map");
    CK(cudaMemset(t.sky, 0, b));
  }
  if (t.mesh) {
    const size_t b = 8 * (size_t)t.mesh * t.mesh * t.mesh;
    if (dev_alloc((void**)&t.grid, b) != cudaSuccess) {
      if (t.sky) cudaFree(t.sky);
      return fail(c, DZS_ENOMEM, "3D lightcone grid");
    }
    CK(cudaMemset(t.grid, 0, b));
  }
  c->obs = t;
  return DZS_OK;
}

dzs_status dzs_observe_add_records(dzs_ctx* c, const dzs_lc_record* rec, size_t n) {
  dzs_status s = guard(c);
  if (s) return s;
  if (n && !rec) return fail(c, DZS_EINVAL, "rec is NULL");
  if (!c->obs.sky && !c->obs.grid) return fail(c, DZS_ESTATE, "observables are off");
  // staged through the conversion scratch (24 cap bytes), in chunks
  const size_t chunk = (size_t)(24 * c->cap) / sizeof(dzs_lc_record);
  dzs_lc_record* d = (dzs_lc_record*)c->B.convert;
  for (size_t done = 0; done < n;) {
    const size_t m = n - done < chunk ? n - done : chunk;
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpy(d, rec + done, m * sizeof(dzs_lc_record), cudaMemcpyHostToDevice));
    launch_observe_records(c, d, (int64_t)m);
    done += m;
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));
  return check_device_errors(c);
}

dzs_status dzs_skymap_get(dzs_ctx* c, uint64_t* map, size_t npix) {
  dzs_status s = guard(c);
  if (s) return s;
  if (!c->obs.sky || !map || npix != (size_t)(12 * c->obs.nside * c->obs.nside))
    return fail(c, DZS_EINVAL, "sky map off or npix != 12 nside^2");
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(map, c->obs.sky, 8 * npix, cudaMemcpyDeviceToHost));
  return DZS_OK;
}

dzs_status dzs_lcdensity_get(dzs_ctx* c, uint64_t* grid, size_t ncell) {
  dzs_status s = guard(c);
  if (s) return s;
  if (!c->obs.grid || !grid || ncell != (size_t)(c->obs.mesh * c->obs.mesh * c->obs.mesh))
    return fail(c, DZS_EINVAL, "3D lightcone grid off or ncell != mesh^3");
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(grid, c->obs.grid, 8 * ncell, cudaMemcpyDeviceToHost));
  return DZS_OK;
}

dzs_status dzs_skymap_alm(dzs_ctx* c, int32_t lmax, double* cl, double* alm) {
  dzs_status s = guard(c);
  if (s) return s;
  if (!c->obs.sky) return fail(c, DZS_ESTATE, "sky map off");
  if (lmax < 0 || lmax > 4 * c->obs.nside || !cl) return fail(c, DZS_EINVAL, "need 0 <= lmax <= 4 nside, cl");
  const size_t need = sht_work_bytes(c->obs.nside, lmax);
  CK(cudaStreamSynchronize(c->stream));
  if (c->sht_bytes < need) {
    if (c->sht_work) CK(cudaFree(c->sht_work));
    c->sht_work = nullptr;
    c->sht_bytes = 0;
    if (dev_alloc(&c->sht_work, need) != cudaSuccess) return fail(c, DZS_ENOMEM, "harmonic-analysis scratch");
    c->sht_bytes = need;
  }
  double2* d_alm = nullptr;
  double* d_cl = nullptr;
  launch_sht(c, lmax, c->sht_work, &d_alm, &d_cl);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(cl, d_cl, 8 * ((size_t)lmax + 1), cudaMemcpyDeviceToHost));
  if (alm) CK(cudaMemcpy(alm, d_alm, 16 * ((size_t)lmax + 1) * (lmax + 2) / 2, cudaMemcpyDeviceToHost));
  return check_device_errors(c);
}

dzs_status dzs_power_spectrum(dzs_ctx* c, int32_t nbins, int32_t flags, double* k, double* pk, double* nmodes) {
  dzs_status s = guard(c);
  if (s) return s;
  if (!c->have_state) return fail(c, DZS_ESTATE, "no particle state");
  if (nbins < 1 || nbins > c->M / 2 || !pk || (flags & ~DZS_PK_SHOT))
    return fail(c, DZS_EINVAL, "need 1 <= nbins <= mesh / 2, pk, known flags");
  // shot noise L^3 sum k^2 / (sum k)^2; sum k = N0 (mass is conserved exactly)
  unsigned long long* k2 = (unsigned long long*)(c->B.counters + 15);
  launch_sum_k2(c, k2);
  unsigned long long sk2 = 0;
  CK(cudaMemcpyAsync(&sk2, k2, sizeof sk2, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const double L = c->P.box, n0 = (double)c->N0;
  const double shot = (flags & DZS_PK_SHOT) ? L * L * L * (double)sk2 / (n0 * n0) : 0.0;
  // CIC needs the Morton order: sort, bin, then put the state back in its order
  // (g is not moved by either, so it stays with its particles)
  double* part = (double*)c->B.phi;  // mesh scratch: M nbins 3 + nbins 3 doubles
  double* out = part + (size_t)c->M * nbins * 3;
  launch_keys(c);
  launch_sort(c);
  launch_pk(c, nbins, part, out, shot);
  std::vector<double> h((size_t)nbins * 3);
  CK(cudaMemcpyAsync(h.data(), out, 8 * h.size(), cudaMemcpyDeviceToHost, c->stream));
  launch_unpermute(c, (double*)c->B.convert);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));
  for (int b = 0; b < nbins; ++b) {
    const double cnt = h[3 * b];
    if (nmodes) nmodes[b] = cnt;
    if (k) k[b] = cnt > 0 ? h[3 * b + 1] / cnt : 0.0;
    pk[b] = cnt > 0 ? h[3 * b + 2] / cnt : 0.0;
  }
  return check_device_errors(c);
}

dzs_status dzs_fof(dzs_ctx* c, double link, int32_t nmin, dzs_halo* halos, size_t cap, size_t* nhalo,
                   int64_t* label) {
  dzs_status s = guard(c);
  if (s) return s;
  if (!c->have_state) return fail(c, DZS_ESTATE, "no particle state");
  if (!(link > 0) || !(link * c->P.box / c->P.n1d < 0.25 * c->P.box) || nmin < 2 || !nhalo || (cap && !halos))
    return fail(c, DZS_EINVAL, "need 0 < link lambda < L / 4, nmin >= 2, nhalo");
  // friends: d^2 <= floor((link 2^32 / n1d)^2) (FP64, then integer)
  const double lb = link * 4294967296.0 / (double)c->P.n1d;
  const uint64_t T = (uint64_t)std::floor(lb * lb);
  // the finest cell depth <= log2 M whose side exceeds the linking length
  int depth = c->logM;
  while (depth > 1 && std::ldexp(1.0, 32 - depth) * std::ldexp(1.0, 32 - depth) < (double)T + 1.0) --depth;
  // work on the Morton order, then put the state back in its order
  launch_keys(c);
  launch_sort(c);
  dzs_halo* d_h = nullptr;
  int64_t* d_label = label ? (int64_t*)c->B.key2 : nullptr;
  launch_fof(c, depth, T, nmin, d_label, &d_h);
  int32_t nh = 0;
  CK(cudaMemcpyAsync(&nh, c->B.n + 2, sizeof nh, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  s = check_device_errors(c);
  if (s) return s;
  std::vector<dzs_halo> h((size_t)nh);
  if (nh) CK(cudaMemcpy(h.data(), d_h, sizeof(dzs_halo) * (size_t)nh, cudaMemcpyDeviceToHost));
  size_t n = 0;
  CK(cudaMemcpy(&n, c->B.n, sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (label) CK(cudaMemcpy(label, d_label, sizeof(int64_t) * (size_t)(int32_t)n, cudaMemcpyDeviceToHost));
  launch_unpermute(c, (double*)c->B.convert);
  CK(cudaGetLastError());
  std::sort(h.begin(), h.end(), [](const dzs_halo& a, const dzs_halo& b) { return a.first < b.first; });
  *nhalo = (size_t)nh;
  for (size_t i = 0; i < h.size() && i < cap; ++i) halos[i] = h[i];
  return check_device_errors(c);
}

dzs_status dzs_get_tables(dzs_ctx* c, double* a, double* drift, double* kick1, double* kick2, double* rlc,
                          uint64_t* rlat) {
  if (!c) return DZS_EINVAL;
  size_t ns = (size_t)c->P.nsteps;
  if (a) memcpy(a, c->T.a.data(), 8 * (ns + 1));
  if (drift) memcpy(drift, c->T.drift.data(), 8 * ns);
  if (kick1) memcpy(kick1, c->T.kick1.data(), 8 * ns);
  if (kick2) memcpy(kick2, c->T.kick2.data(), 8 * ns);
  if (rlc) memcpy(rlc, c->T.rlc.data(), 8 * (ns + 1));
  if (rlat) memcpy(rlat, c->T.rlat.data(), 8 * (ns + 1));
  return DZS_OK;
}

dzs_status dzs_get_mesh(dzs_ctx* c, int32_t which, double* out) {
  dzs_status s = guard(c);
  if (s) return s;
  if (!out || (which != DZS_MESH_DELTA && which != DZS_MESH_PHI)) return fail(c, DZS_EINVAL, "bad arguments");
  s = check_device_errors(c);
  if (s) return s;
  int64_t m3 = (int64_t)c->M * c->M * c->M;
  const void* src = which == DZS_MESH_DELTA ? c->B.rho : c->B.phi;
  if (c->fp64) {
    CK(cudaMemcpy(out, src, 8 * m3, cudaMemcpyDeviceToHost));
  } else {
    float* tmp = new (std::nothrow) float[m3];
    if (!tmp) return fail(c, DZS_ENOMEM, "host buffer");
    cudaError_t e = cudaMemcpy(tmp, src, 4 * m3, cudaMemcpyDeviceToHost);
    for (int64_t i = 0; i < m3 && e == cudaSuccess; ++i) out[i] = tmp[i];
    delete[] tmp;
    if (e != cudaSuccess) return fail(c, DZS_ECUDA, "mesh copy", cudaGetErrorString(e));
  }
  return DZS_OK;
}

dzs_status dzs_set_profiling(dzs_ctx* c, int32_t enable) {
  dzs_status s = guard(c);
  if (s) return s;
  CK(cudaStreamSynchronize(c->stream));
  for (auto& pe : c->prof_pending) {
    c->ev_pool.push_back(pe.a);
    c->ev_pool.push_back(pe.b);
  }
  c->prof_pending.clear();
  for (int i = 0; i < 8; ++i) {
    c->prof_ms[i] = 0;
    c->prof_calls[i] = 0;
  }
  CK(cudaMemsetAsync(c->B.counters + 4, 0, 4 * sizeof(uint64_t), c->stream));
  CK(cudaMemsetAsync(c->B.counters + 12, 0, 2 * sizeof(uint64_t), c->stream));
  CK(cudaMemsetAsync(c->B.counters + 20, 0, 2 * sizeof(uint64_t), c->stream));
  c->prof_on = (enable & DZS_PROFILE_STAGES) != 0;
  c->walk_diag = (enable & DZS_PROFILE_WALK) != 0;
  return DZS_OK;
}

dzs_status dzs_get_profile(dzs_ctx* c, double ms[DZS_PROF_N], uint64_t calls[DZS_PROF_N]) {
  dzs_status s = guard(c);
  if (s) return s;
  CK(cudaStreamSynchronize(c->stream));
  for (auto& pe : c->prof_pending) {
    float t = 0;
    CK(cudaEventElapsedTime(&t, pe.a, pe.b));
    c->prof_ms[pe.cat] += t;
    c->prof_calls[pe.cat] += 1;
    c->ev_pool.push_back(pe.a);
    c->ev_pool.push_back(pe.b);
  }
  c->prof_pending.clear();
  for (int i = 0; i < DZS_PROF_N; ++i) {
    if (ms) ms[i] = c->prof_ms[i];
    if (calls) calls[i] = c->prof_calls[i];
  }
  return DZS_OK;
}

dzs_status dzs_get_counters(dzs_ctx* c, uint64_t out[9]) {
  dzs_status s = guard(c);
  if (s) return s;
  if (!out) return fail(c, DZS_EINVAL, "out is NULL");
  CK(cudaStreamSynchronize(c->stream));
  uint64_t ctr[16];
  uint32_t err = 0;
  CK(cudaMemcpy(ctr, c->B.counters, sizeof ctr, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&err, c->B.err, sizeof err, cudaMemcpyDeviceToHost));
  out[0] = ctr[2];
  out[1] = ctr[3];
  out[2] = ctr[4];
  out[3] = err;
  out[4] = c->launches;
  out[5] = ctr[0];
  out[6] = ctr[7];
  out[7] = ctr[12];
  out[8] = ctr[13];
  return DZS_OK;
}

void dzs_debug_fail_alloc(int32_t k) { g_fail_alloc.store(k > 0 ? k : 0); }

dzs_status dzs_twin_displacement(dzs_ctx* a, dzs_ctx* b, const double* edges, int32_t nbins, uint64_t* counts,
                                 uint64_t* matched, double* max_ratio) {
  dzs_status s = guard(a);
  if (s) return s;
  s = guard(b);
  if (s) return s;
  if (!edges || nbins < 1 || !counts) return fail(a, DZS_EINVAL, "edges, nbins or counts");
  for (int k = 0; k < nbins; ++k)
    if (!(edges[k] < edges[k + 1])) return fail(a, DZS_EINVAL, "edges must increase");
  if (a->dev != b->dev || a->N0 != b->N0 || a->P.box != b->P.box)
    return fail(a, DZS_EINVAL, "twin runs must share the device, N0 and the box");
  if (!a->have_state || !b->have_state) return fail(a, DZS_ESTATE, "no particle state");
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return fail(b, DZS_EDEVICE, "device failure");
  const size_t bytes = 4 * (size_t)a->N0 + 8 * (size_t)(nbins + 1) + 8 * (size_t)nbins + 16 + 1024;
  char* tmp = nullptr;
  if (dev_alloc((void**)&tmp, bytes) != cudaSuccess) return fail(a, DZS_ENOMEM, "twin displacement scratch");
  double* d_edges = (double*)tmp;
  unsigned long long* d_counts = (unsigned long long*)(tmp + 8 * (size_t)(nbins + 1));
  unsigned long long* d_stats = d_counts + nbins;
  int32_t* map = (int32_t*)(d_stats + 2);
  dzs_status st = DZS_OK;
  if (cudaMemcpyAsync(d_edges, edges, 8 * (size_t)(nbins + 1), cudaMemcpyHostToDevice, a->stream) != cudaSuccess ||
      cudaMemsetAsync(d_counts, 0, 8 * (size_t)(nbins + 2), a->stream) != cudaSuccess) {
    st = fail(a, DZS_ECUDA, "twin displacement set-up");
  }
  if (!st) {
    const double h = a->P.box / a->P.n1d / 40.0;  // softening length of Sec. 3.2
    launch_twin_displacement(a, b, map, d_edges, nbins, h, d_counts, d_stats);
    std::vector<unsigned long long> hc((size_t)nbins + 2);
    if (cudaMemcpyAsync(hc.data(), d_counts, 8 * hc.size(), cudaMemcpyDeviceToHost, a->stream) != cudaSuccess ||
        cudaStreamSynchronize(a->stream) != cudaSuccess) {
      st = fail(a, DZS_EDEVICE, "twin displacement");
    } else {
      for (int k = 0; k < nbins; ++k) counts[k] = hc[k];
      if (matched) *matched = hc[nbins];
      if (max_ratio) {
        const unsigned long long bits = hc[nbins + 1];
        double v;
        std::memcpy(&v, &bits, 8);
        *max_ratio = v;
      }
    }
  }
  cudaFree(tmp);
  return st;
}

dzs_status dzs_get_walk_counters(dzs_ctx* c, uint64_t out[6]) {
  dzs_status s = guard(c);
  if (s) return s;
  if (!out) return fail(c, DZS_EINVAL, "out is NULL");
  CK(cudaStreamSynchronize(c->stream));
  uint64_t ctr[22];
  CK(cudaMemcpy(ctr, c->B.counters, sizeof ctr, cudaMemcpyDeviceToHost));
  out[0] = ctr[4];
  out[1] = ctr[5];
  out[2] = ctr[12];
  out[3] = ctr[13];
  out[4] = ctr[20];
  out[5] = ctr[21];
  return DZS_OK;
}

dzs_status dzs_walk_lists(dzs_ctx* c, int64_t* first, int64_t* count, int64_t* list_len, size_t cap,
                          size_t* ngroups) {
  dzs_status s = guard(c);
  if (s) return s;
  if (!ngroups) return fail(c, DZS_EINVAL, "ngroups is NULL");
  CK(cudaStreamSynchronize(c->stream));
  uint64_t ng = 0;
  CK(cudaMemcpy(&ng, c->B.counters + 2, sizeof ng, cudaMemcpyDeviceToHost));
  *ngroups = (size_t)ng;
  if (!first && !count && !list_len) return DZS_OK;
  if (cap < ng) return fail(c, DZS_EINVAL, "cap is below the number of walk groups");
  std::vector<int32_t> gidx(ng), glen(ng);
  std::vector<dzs::Node> nodes;
  if (ng) {
    CK(cudaMemcpy(gidx.data(), c->B.groups, 4 * ng, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(glen.data(), c->B.wlen, 4 * ng, cudaMemcpyDeviceToHost));
    int32_t maxi = 0;
    for (int32_t g : gidx) maxi = g > maxi ? g : maxi;
    nodes.resize((size_t)maxi + 1);
    CK(cudaMemcpy(nodes.data(), c->B.nodes, sizeof(dzs::Node) * nodes.size(), cudaMemcpyDeviceToHost));
  }
  for (uint64_t g = 0; g < ng; ++g) {
    const dzs::Node& nd = nodes[gidx[g]];
    if (first) first[g] = nd.start;
    if (count) count[g] = nd.count;
    if (list_len) list_len[g] = glen[g];
  }
  return DZS_OK;
}

const char* dzs_last_error(const dzs_ctx* c) {
  if (!c) return g_create_error.c_str();
  return c->err.c_str();
}

}  // extern "C"
