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
  int lockstep = 0;  // > 0: that many workers, each stepping its resident runs as one lockstep group
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

// A request resident in the lockstep group.
struct Resident {
  Req* r = nullptr;
  vp_sim* sim = nullptr;
  int done = 0;
};

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

// Retire a resident run: its final state (keep_f) and its record.
void retire(vp_batch* b, vp_ctx* ctx, vp_group* g, Resident& rs, int status) {
  Req* r = rs.r;
  if (status == VP_OK && r->keep_f) {
    r->fT.resize((size_t)1 << (r->lay.nx + r->lay.nv));
    status = mps_to_grid(ctx, vp_sim_state(rs.sim), &r->lay, r->fT.data());
  }
  if (rs.sim) {
    if (g) vp_group_remove(g, rs.sim);
    vp_sim_destroy(rs.sim);
  }
  r->recs.resize(rs.done);
  r->step_ms.resize(rs.done);
  r->status = status;
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

// Continuous batching in lockstep: between group steps, runs that finished
// or failed leave the group and pending requests join it while slots and
// memory allow; every group step advances all resident runs with batched
// launches (vp_group_step).  A run's per-step latency is the group step's.
// With several lockstep workers, each keeps a group of runs with the same
// number of sites (its key, taken from the first run it admits while empty):
// runs of one size step together, and the groups of different sizes overlap
// on the device.  Requests are taken first-in first-out among those that
// match the worker's key and fit the budget.
int site_count(const Req* r) { return r->lay.nx + r->lay.nv; }

void lockstep_loop(vp_batch* b, int w) {
  vp_ctx* ctx = b->wctx[w];
  cudaSetDevice(ctx->device);
  vp_group* g = nullptr;
  if (vp_group_create(ctx, b->max_conc, &g) != VP_OK) g = nullptr;
  std::vector<Resident> res;
  int key = -1;  // site count of this worker's runs (-1: none resident)
  auto admissible = [&](std::deque<Req*>& q) {
    for (auto it = q.begin(); it != q.end(); ++it)
      if ((key < 0 || site_count(*it) == key) && b->in_use + (*it)->footprint <= b->budget) return it;
    return q.end();
  };
  for (;;) {
    std::vector<Req*> admit;
    {
      std::unique_lock<std::mutex> lk(b->mu);
      b->cv.wait(lk, [&] { return b->stop || !res.empty() || admissible(b->pending) != b->pending.end(); });
      if (b->stop) break;
      for (;;) {
        if ((int)(res.size() + admit.size()) >= b->max_conc) break;
        auto it = admissible(b->pending);
        if (it == b->pending.end()) break;
        Req* r = *it;
        b->pending.erase(it);
        b->in_use += r->footprint;
        b->active++;
        key = site_count(r);
        admit.push_back(r);
      }
    }
    // the admitted runs' initial MPS in one batched decomposition
    const int na = (int)admit.size();
    std::vector<vp_layout> lays(na);
    std::vector<const double*> fs(na);
    std::vector<int> chis(na), cst(na, VP_OK);
    std::vector<double> tols(na);
    std::vector<mps_t*> ms(na, nullptr);
    for (int a = 0; a < na; ++a) {
      admit[a]->t_start = now_ms();
      lays[a] = admit[a]->lay;
      fs[a] = admit[a]->f0.data();
      chis[a] = admit[a]->cfg.chi;
      tols[a] = admit[a]->cfg.tol;
    }
    int gst = g ? VP_OK : VP_ENOMEM;
    if (gst == VP_OK && na > 0)
      gst = vp_group_mps_create(g, na, lays.data(), fs.data(), chis.data(), tols.data(), ms.data(), cst.data());
    for (int a = 0; a < na; ++a) {
      Req* r = admit[a];
      Resident rs;
      rs.r = r;
      r->recs.resize(r->nsteps);
      r->step_ms.resize(r->nsteps);
      mps_t* m = ms[a];
      int st = gst != VP_OK ? gst : cst[a];
      if (st == VP_OK) st = vp_sim_create(ctx, &r->lay, &r->cfg, m, &rs.sim);
      if (m) mps_destroy(m);
      if (st == VP_OK && r->nsteps > 0) st = vp_group_add(g, rs.sim);
      r->f0.clear();
      r->f0.shrink_to_fit();
      if (st != VP_OK || r->nsteps == 0) {
        if (st != VP_OK && rs.sim) {
          vp_sim_destroy(rs.sim);
          rs.sim = nullptr;
        }
        retire(b, ctx, nullptr, rs, st);
        continue;
      }
      res.push_back(rs);
    }
    if (res.empty()) {
      key = -1;
      continue;
    }
    std::vector<vp_record> recs(res.size());
    std::vector<int> status(res.size(), VP_OK);
    const double t0 = now_ms();
    const int st = vp_group_step(g, recs.data(), status.data());
    const double dt_ms = now_ms() - t0;
    std::vector<Resident> keep;
    for (size_t i = 0; i < res.size(); ++i) {
      Resident& rs = res[i];
      int si = st != VP_OK ? st : status[i];
      if (si == VP_OK) {
        rs.r->recs[rs.done] = recs[i];
        rs.r->step_ms[rs.done] = dt_ms;
        rs.done++;
      }
      if (si != VP_OK || rs.done >= rs.r->nsteps)
        retire(b, ctx, g, rs, si);
      else
        keep.push_back(rs);
    }
    res.swap(keep);
    if (res.empty()) key = -1;
  }
  for (Resident& rs : res) retire(b, ctx, g, rs, VP_EBUSY);
  if (g) vp_group_destroy(g);
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
  if (!parent || !out || max_concurrent < 1 || max_concurrent > 4096 || mem_budget_bytes == 0) return VP_EINVAL;
  vp_batch* b = new vp_batch();
  b->parent = parent;
  b->max_conc = max_concurrent;
  b->budget = mem_budget_bytes;
  *out = b;
  return VP_OK;
}

// Worker contexts, each with its own stream: one per worker thread, or one
// for the lockstep worker (whose grid-cooperative kernels may use every SM).
static int make_workers(vp_batch* b) {
  vp_ctx* parent = b->parent;
  const int nw = b->lockstep ? b->lockstep : b->max_conc;
  if (!b->lockstep && nw > 64) return vp::fail(parent, VP_EINVAL, "vp_batch: at most 64 worker threads");
  for (int w = 0; w < nw; ++w) {
    cudaStream_t st = nullptr;
    vp_ctx* c = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        vp_ctx_create(st, nullptr, nullptr, nullptr, &c) != VP_OK) {
      if (st) cudaStreamDestroy(st);
      for (vp_ctx* x : b->wctx) vp_ctx_destroy(x);
      b->wctx.clear();
      return vp::fail(parent, VP_ECUDA, "vp_batch_start: worker context failed");
    }
    c->owns_stream = true;
    c->coop_cap = std::max(16, parent->num_sms / nw);
    c->wait_clocks = parent->wait_clocks;
    if (vp::write_wait_limit(c) != VP_OK) {
      vp_ctx_destroy(c);
      for (vp_ctx* x : b->wctx) vp_ctx_destroy(x);
      b->wctx.clear();
      return vp::fail(parent, VP_ECUDA, "vp_batch_start: worker context failed");
    }
    b->wctx.push_back(c);
  }
  return VP_OK;
}

int vp_batch_set_lockstep(vp_batch* b, int groups) {
  if (!b || groups < 0 || groups > 16) return VP_EINVAL;
  std::lock_guard<std::mutex> lk(b->mu);
  if (b->started) return vp::fail(b->parent, VP_EBUSY, "vp_batch_set_lockstep: workers already started");
  b->lockstep = groups;
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
  VP_TRY(make_workers(b));
  b->started = true;
  if (b->lockstep)
    for (int w = 0; w < b->lockstep; ++w) b->workers.emplace_back(lockstep_loop, b, w);
  else
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

int64_t vp_batch_kernel_launches(const vp_batch* b) {
  if (!b) return 0;
  int64_t n = 0;
  for (const vp_ctx* c : b->wctx) n += vp_kernel_launches(c);
  return n;
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
