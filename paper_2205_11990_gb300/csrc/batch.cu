// Many independent simulations on one GPU: a pool of host worker threads,
// each with its own library context (own CUDA stream, stream-ordered
// allocator, device status words).  Requests are admitted first-in first-out
// when a worker is free and their memory footprint fits the budget; requests
// submitted while others run join as slots free up (continuous batching), and
// the kernels of co-resident runs overlap on the device.  Each run's results
// do not depend on what else is running: every run keeps its own buffers,
// scratch and stream, and the arithmetic is deterministic.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
  uint64_t id = 0;
  vp_layout lay{};
  vp_config cfg{};
  std::vector<double> f0;
  int nsteps = 0;
  int keep_f = 0;
  size_t footprint = 0;
  int status = VP_OK;
  std::vector<vp_record> recs;
  std::vector<double> step_ms;
  std::vector<double> fT;
  double t_submit = 0, t_start = 0, t_end = 0;
  bool polled = false;
  bool done = false;
};

double quantile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * (double)(v.size() - 1);
  const size_t lo = (size_t)pos;
  const size_t hi = std::min(v.size() - 1, lo + 1);
  return v[lo] + (pos - (double)lo) * (v[hi] - v[lo]);
}

}  // namespace

struct vp_batch {
  vp_ctx* parent = nullptr;
  int max_conc = 1;
  size_t budget = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req*> pending;
  std::map<uint64_t, Req*> all;
  size_t in_use = 0;
  int active = 0;
  int unfinished = 0;
  bool stop = false;
  bool started = false;
  uint64_t next_id = 1;
  std::vector<std::thread> workers;
  std::vector<vp_ctx*> wctx;
};

extern "C" int vp_ctx_create(void* cuda_stream, vp_alloc_fn alloc, vp_free_fn free_fn, void* user, vp_ctx** out);

namespace {

void run_request(vp_ctx* ctx, Req* r) {
  mps_t* m = nullptr;
  vp_sim* sim = nullptr;
  int st = mps_create(ctx, &r->lay, r->f0.data(), 0, r->cfg.chi, r->cfg.tol, &m);
  if (st == VP_OK) st = vp_sim_create(ctx, &r->lay, &r->cfg, m, &sim);
  if (m) mps_destroy(m);
  r->recs.resize(r->nsteps);
  r->step_ms.resize(r->nsteps);
  for (int i = 0; st == VP_OK && i < r->nsteps; ++i) {
    const double t0 = now_ms();
    st = vp_step(sim, 1, &r->recs[i]);
    r->step_ms[i] = now_ms() - t0;
  }
  if (st == VP_OK && r->keep_f) {
    r->fT.resize((size_t)1 << (r->lay.nx + r->lay.nv));
    st = mps_to_grid(ctx, vp_sim_state(sim), &r->lay, r->fT.data());
  }
  if (sim) vp_sim_destroy(sim);
  r->f0.clear();
  r->f0.shrink_to_fit();
  r->status = st;
}

void worker_loop(vp_batch* b, int w) {
  vp_ctx* ctx = b->wctx[w];
  cudaSetDevice(ctx->device);
  for (;;) {
    Req* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(b->mu);
      b->cv.wait(lk, [&] {
        return b->stop || (!b->pending.empty() && b->in_use + b->pending.front()->footprint <= b->budget);
      });
      if (b->stop) return;
      r = b->pending.front();
      b->pending.pop_front();
      b->in_use += r->footprint;
      b->active++;
    }
    r->t_start = now_ms();
    run_request(ctx, r);
    r->t_end = now_ms();
    {
      std::lock_guard<std::mutex> lk(b->mu);
      b->in_use -= r->footprint;
      b->active--;
      b->unfinished--;
      r->done = true;
    }
    b->cv.notify_all();
  }
}

}  // namespace

extern "C" {

size_t vp_footprint_bytes(const vp_layout* L, const vp_config* cfg) {
  if (!L || !cfg) return 0;
  const int n = L->nx + L->nv;
  const int W = 12;                                  // operator bond (sequential map, field bond ~8)
  const size_t cap = (size_t)std::max(1, cfg->chi) * 3;  // tolerance-compressed bonds stay within ~3 chi
  size_t states = 0, worst = 0;
  for (int k = 0; k < n; ++k) {
    const size_t full_l = (size_t)1 << std::min(k, n - k), full_r = (size_t)1 << std::min(k + 1, n - k - 1);
    const size_t rl = std::min(full_l, cap), rr = std::min(full_r, cap);
    states += 16 * rl * rr;                           // one core, bytes
    worst = std::max(worst, 16 * (rl * W + rl) * (rr * W + rr));
  }
  // f, fi, acc, two sums (pre-compression), factorisation workspaces
  return 3 * states + 2 * worst + 4 * worst + ((size_t)8 << (n + 1)) + ((size_t)64 << 20);
}

int vp_batch_create(vp_ctx* parent, int max_concurrent, size_t mem_budget_bytes, vp_batch** out) {
  if (!parent || !out || max_concurrent < 1 || max_concurrent > 64 || mem_budget_bytes == 0) return VP_EINVAL;
  vp_batch* b = new vp_batch();
  b->parent = parent;
  b->max_conc = max_concurrent;
  b->budget = mem_budget_bytes;
  for (int w = 0; w < max_concurrent; ++w) {
    cudaStream_t st = nullptr;
    vp_ctx* c = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        vp_ctx_create(st, nullptr, nullptr, nullptr, &c) != VP_OK) {
      if (st) cudaStreamDestroy(st);
      for (vp_ctx* x : b->wctx) vp_ctx_destroy(x);
      delete b;
      return vp::fail(parent, VP_ECUDA, "vp_batch_create: worker context failed");
    }
    c->owns_stream = true;
    c->coop_cap = std::max(16, parent->num_sms / max_concurrent);
    b->wctx.push_back(c);
  }
  *out = b;
  return VP_OK;
}

int vp_batch_submit(vp_batch* b, const vp_layout* L, const vp_config* cfg, const double* f0, int nsteps, int keep_f,
                    uint64_t* id_out) {
  if (!b || !L || !cfg || !f0 || nsteps < 0) return VP_EINVAL;
  const size_t fp = vp_footprint_bytes(L, cfg);
  if (fp > b->budget) return vp::fail(b->parent, VP_ECAPACITY, "vp_batch_submit: footprint exceeds the budget");
  Req* r = new Req();
  r->lay = *L;
  r->cfg = *cfg;
  r->cfg.streams = 1;  // runs overlap each other; no second stream per run
  r->nsteps = nsteps;
  r->keep_f = keep_f;
  r->footprint = fp;
  r->f0.assign(f0, f0 + ((size_t)1 << (L->nx + L->nv)));
  r->t_submit = now_ms();
  {
    std::lock_guard<std::mutex> lk(b->mu);
    r->id = b->next_id++;
    b->all[r->id] = r;
    b->pending.push_back(r);
    b->unfinished++;
  }
  b->cv.notify_all();
  if (id_out) *id_out = r->id;
  return VP_OK;
}

int vp_batch_start(vp_batch* b) {
  if (!b) return VP_EINVAL;
  std::lock_guard<std::mutex> lk(b->mu);
  if (b->started) return VP_OK;
  b->started = true;
  for (int w = 0; w < b->max_conc; ++w) b->workers.emplace_back(worker_loop, b, w);
  return VP_OK;
}

int vp_batch_wait(vp_batch* b) {
  if (!b) return VP_EINVAL;
  std::unique_lock<std::mutex> lk(b->mu);
  if (!b->started) return VP_EINVAL;
  b->cv.wait(lk, [&] { return b->unfinished == 0; });
  return VP_OK;
}

int vp_batch_poll(vp_batch* b, vp_result* out, int max, int* n_out) {
  if (!b || (!out && max > 0) || !n_out) return VP_EINVAL;
  std::lock_guard<std::mutex> lk(b->mu);
  int n = 0;
  for (auto& kv : b->all) {
    Req* r = kv.second;
    if (n >= max) break;
    if (!r->done || r->polled) continue;
    r->polled = true;
    vp_result& o = out[n++];
    std::memset(&o, 0, sizeof(o));
    o.id = r->id;
    o.status = r->status;
    o.nsteps = r->nsteps;
    o.queue_ms = r->t_start - r->t_submit;
    o.run_ms = r->t_end - r->t_start;
    o.step_ms_p50 = quantile(r->step_ms, 0.5);
    o.step_ms_p99 = quantile(r->step_ms, 0.99);
    o.field_energy = r->recs.empty() ? 0.0 : r->recs.back().field_energy;
    int mb = 0;
    for (auto& rc : r->recs) mb = std::max(mb, rc.max_bond);
    o.max_bond = mb;
  }
  *n_out = n;
  return VP_OK;
}

int vp_batch_records(vp_batch* b, uint64_t id, vp_record* records, double* step_ms, double* fT) {
  if (!b) return VP_EINVAL;
  std::lock_guard<std::mutex> lk(b->mu);
  auto it = b->all.find(id);
  if (it == b->all.end() || !it->second->done) return VP_EINVAL;
  Req* r = it->second;
  if (records) std::copy(r->recs.begin(), r->recs.end(), records);
  if (step_ms) std::copy(r->step_ms.begin(), r->step_ms.end(), step_ms);
  if (fT) {
    if (r->fT.empty()) return VP_EINVAL;
    std::copy(r->fT.begin(), r->fT.end(), fT);
  }
  return VP_OK;
}

int vp_batch_destroy(vp_batch* b) {
  if (!b) return VP_EINVAL;
  {
    std::lock_guard<std::mutex> lk(b->mu);
    b->stop = true;
  }
  b->cv.notify_all();
  for (auto& t : b->workers) t.join();
  for (vp_ctx* c : b->wctx) vp_ctx_destroy(c);
  for (auto& kv : b->all) delete kv.second;
  delete b;
  return VP_OK;
}

}  // extern "C"
