// serve.cu -- continuous batching of lightcone-mock requests on one GPU.
//
// Requests arrive over time (Poisson stream or any schedule); each becomes a
// context of its own, with its own non-blocking CUDA stream and its state
// resident in HBM, admitted in arrival order as soon as the sum of the
// admitted contexts' footprints (dzs_footprint_bytes) stays within the HBM
// budget.  Several host threads share the work: each admits the next request
// when it has arrived and fits, and keeps its own mocks' streams fed with
// slices of steps (at most two slices in flight, each closed by an event), so
// mocks of different sizes overlap on the device and the kernel launches of
// small mocks are issued in parallel; a finished mock is drained, hashed and
// destroyed, which frees its memory for the next admission.
// Contexts share nothing, and every reduction of the step is deterministic,
// so a mock's result does not depend on what runs beside it.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "common.cuh"

namespace {

struct Active {
  size_t req = 0;
  dzs_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  size_t bytes = 0;
  int32_t enqueued = 0;  // steps enqueued so far
  int32_t nsteps = 0;
  std::deque<cudaEvent_t> inflight;
};

uint64_t fnv1a(const void* data, size_t len, uint64_t h) {
  const unsigned char* p = (const unsigned char*)data;
  for (size_t i = 0; i < len; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

}  // namespace

// ---- a batch of contexts stepped together: each host worker thread enqueues
// the steps of its share of the contexts in slices, so every stream gets
// work early and the launches of many small mocks are issued in parallel.
// The contexts stay the caller's; results do not depend on the batch.
struct dzs_batch {
  std::vector<dzs_ctx*> ctx;
  int threads = 1;
};

extern "C" dzs_status dzs_batch_create(dzs_ctx* const* ctxs, int32_t n, int32_t host_threads, dzs_batch** out) {
  if (!out || n < 0 || (n > 0 && !ctxs) || host_threads < 0) return DZS_EINVAL;
  *out = nullptr;
  for (int32_t i = 0; i < n; ++i)
    if (!ctxs[i]) return DZS_EINVAL;
  dzs_batch* b = new (std::nothrow) dzs_batch();
  if (!b) return DZS_ENOMEM;
  b->ctx.assign(ctxs, ctxs + n);
  int t = host_threads;
  if (t == 0) {
    const unsigned hw = std::thread::hardware_concurrency();
    t = (int)std::min(8u, hw > 0 ? hw : 1u);
  }
  b->threads = std::max(1, std::min(t, std::max(1, (int)n)));
  *out = b;
  return DZS_OK;
}

extern "C" dzs_status dzs_batch_step(dzs_batch* b, int32_t nsteps, int32_t slice, int32_t* steps_done) {
  if (!b || nsteps < 0 || slice < 1) return DZS_EINVAL;
  const size_t n = b->ctx.size();
  std::vector<int32_t> done(n, 0);
  std::atomic<int> first_error{DZS_OK};
  auto work = [&](int t) {
    int dev = -1;
    // round-robin slices over this thread's contexts (t, t + T, t + 2T, ...)
    bool any = true;
    while (any) {
      any = false;
      for (size_t i = (size_t)t; i < n; i += (size_t)b->threads) {
        if (done[i] >= nsteps) continue;
        dzs_ctx* c = b->ctx[i];
        if (c->dev != dev) {
          cudaSetDevice(c->dev);
          dev = c->dev;
        }
        const int32_t k = std::min(slice, nsteps - done[i]);
        int32_t got = 0;
        const dzs_status st = dzs_step(c, k, &got);
        done[i] += got;
        if (st != DZS_OK) {
          int expect = DZS_OK;
          first_error.compare_exchange_strong(expect, (int)st);
          done[i] = nsteps;  // this context stops here
          continue;
        }
        if (got < k) done[i] = nsteps;  // reached a = 1
        any = true;
      }
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < b->threads; ++t) th.emplace_back(work, t);
  work(0);
  for (auto& x : th) x.join();
  if (steps_done)
    for (size_t i = 0; i < n; ++i) steps_done[i] = std::min(done[i], nsteps);
  return (dzs_status)first_error.load();
}

extern "C" dzs_status dzs_batch_synchronize(dzs_batch* b) {
  if (!b) return DZS_EINVAL;
  for (dzs_ctx* c : b->ctx) {
    cudaSetDevice(c->dev);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return DZS_EDEVICE;
  }
  return DZS_OK;
}

extern "C" dzs_status dzs_batch_destroy(dzs_batch* b) {
  delete b;
  return DZS_OK;
}

extern "C" dzs_status dzs_serve(const dzs_serve_config* cfg, const dzs_request* req, size_t n,
                                dzs_request_result* out, double* wall_s) {
  if (!cfg || (n && (!req || !out)) || cfg->steps_per_slice < 1 || !(cfg->hbm_budget_bytes > 0) ||
      cfg->host_threads < 0)
    return DZS_EINVAL;
  using clk = std::chrono::steady_clock;
  const clk::time_point t0 = clk::now();
  auto now = [&]() { return std::chrono::duration<double>(clk::now() - t0).count(); };
  std::vector<size_t> order(n);
  for (size_t i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return req[a].arrival_s < req[b].arrival_s; });
  for (size_t i = 0; i < n; ++i) {
    std::memset(&out[i], 0, sizeof out[i]);
    out[i].status = -1;
  }
  // shared admission state: the next request in arrival order, the memory in
  // use, the number of mocks running and the first error
  std::mutex mu;
  size_t next = 0;
  double used = 0.0;
  int32_t running = 0;
  std::atomic<size_t> finished{0};
  dzs_status first_error = DZS_OK;
  int nthreads = cfg->host_threads;
  if (nthreads == 0) {
    const unsigned hw = std::thread::hardware_concurrency();
    nthreads = (int)std::min(8u, hw > 0 ? hw : 1u);
  }
  nthreads = std::max(1, std::min(nthreads, (int)std::max<size_t>(1, n)));

  auto worker = [&]() {
    cudaSetDevice(cfg->base.device);
    std::vector<Active> act;
    std::vector<cudaEvent_t> pool;
    std::vector<dzs_lc_record> buf;
    auto get_event = [&]() {
      cudaEvent_t e = nullptr;
      if (!pool.empty()) {
        e = pool.back();
        pool.pop_back();
      } else {
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
      }
      return e;
    };
    auto retire = [&](Active& a, dzs_status st) {
      dzs_request_result& r = out[a.req];
      r.status = st;
      if (st == DZS_OK) {
        size_t cnt = 0;
        int32_t step = 0;
        st = dzs_get_count(a.ctx, &cnt, &step);
        r.n_end = cnt;
        if (st == DZS_OK) st = dzs_diagnostics(a.ctx, r.diag);
        uint64_t h = 1469598103934665603ull, total = 0;
        while (st == DZS_OK) {
          size_t got = 0;
          buf.resize(1 << 16);
          st = dzs_lightcone_drain(a.ctx, buf.data(), buf.size(), &got);
          h = fnv1a(buf.data(), got * sizeof(dzs_lc_record), h);
          total += got;
          if (got < buf.size()) break;
        }
        r.records = total;
        r.record_hash = h;
        r.status = st;
      }
      r.done_s = now();
      for (cudaEvent_t e : a.inflight) pool.push_back(e);
      a.inflight.clear();
      dzs_destroy(a.ctx);
      if (a.stream) cudaStreamDestroy(a.stream);
      {
        std::lock_guard<std::mutex> lock(mu);
        used -= (double)a.bytes;
        --running;
        if (st != DZS_OK && first_error == DZS_OK) first_error = st;
      }
      ++finished;
    };
    while (finished.load() < n) {
      bool progress = false;
      // admission: the head of the arrival order, when it has arrived and the
      // budget allows (only the head is ever admitted: arrival order holds)
      for (;;) {
        size_t i = 0, bytes = 0;
        dzs_params p = cfg->base;
        {
          std::lock_guard<std::mutex> lock(mu);
          if (next >= n) break;
          i = order[next];
          if (req[i].arrival_s > now()) break;
          if (cfg->max_active > 0 && running >= cfg->max_active) break;
          p.n1d = req[i].n1d;
          p.mesh = req[i].mesh;
          p.box = req[i].box;
          p.sigma8 = req[i].sigma8;
          p.seed = req[i].seed;
          p.capacity = 0;
          dzs_status st = dzs_footprint_bytes(&p, &bytes);
          if (st == DZS_OK && (double)bytes > cfg->hbm_budget_bytes) st = DZS_ENOMEM;  // never fits
          if (st != DZS_OK) {
            out[i].status = st;
            out[i].admit_s = out[i].done_s = now();
            if (first_error == DZS_OK) first_error = st;
            ++next;
            ++finished;
            progress = true;
            continue;
          }
          if (used + (double)bytes > cfg->hbm_budget_bytes) break;  // wait for memory
          used += (double)bytes;
          ++running;
          ++next;
        }
        Active a;
        a.req = i;
        a.bytes = bytes;
        a.nsteps = p.nsteps;
        cudaStreamCreateWithFlags(&a.stream, cudaStreamNonBlocking);
        dzs_status st = dzs_create(&p, a.stream, &a.ctx);
        out[i].admit_s = now();
        if (st == DZS_OK) st = dzs_ics(a.ctx);
        progress = true;
        if (st != DZS_OK) {
          out[i].status = st;
          out[i].done_s = now();
          if (a.ctx) dzs_destroy(a.ctx);
          if (a.stream) cudaStreamDestroy(a.stream);
          {
            std::lock_guard<std::mutex> lock(mu);
            used -= (double)bytes;
            --running;
            if (first_error == DZS_OK) first_error = st;
          }
          ++finished;
          continue;
        }
        act.push_back(std::move(a));
        break;  // one admission per pass: the other workers get theirs
      }
      // feed this worker's mocks, retire the finished ones
      for (size_t j = 0; j < act.size();) {
        Active& a = act[j];
        while (!a.inflight.empty() && cudaEventQuery(a.inflight.front()) == cudaSuccess) {
          pool.push_back(a.inflight.front());
          a.inflight.pop_front();
          progress = true;
        }
        dzs_status st = DZS_OK;
        while (a.enqueued < a.nsteps && a.inflight.size() < 2) {
          int32_t k = std::min(cfg->steps_per_slice, a.nsteps - a.enqueued), done = 0;
          st = dzs_step(a.ctx, k, &done);
          if (st != DZS_OK) break;
          a.enqueued += k;
          cudaEvent_t e = get_event();
          cudaEventRecord(e, a.stream);
          a.inflight.push_back(e);
          progress = true;
        }
        if (st != DZS_OK || (a.enqueued >= a.nsteps && a.inflight.empty())) {
          retire(a, st);
          act.erase(act.begin() + (std::ptrdiff_t)j);
          progress = true;
          continue;
        }
        ++j;
      }
      if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  };
  std::vector<std::thread> threads;
  for (int t = 1; t < nthreads; ++t) threads.emplace_back(worker);
  worker();
  for (auto& th : threads) th.join();
  if (wall_s) *wall_s = now();
  return first_error;
}
