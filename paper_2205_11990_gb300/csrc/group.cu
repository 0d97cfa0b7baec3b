// Lockstep groups of simulations (vp_group_*): one RK4-C1 step of many
// independent simulations in which every kernel launch serves all members at
// the same position of the step -- the same site of the same sweep of the
// same stage.  The per-site contractions, the QR and the Jacobi SVD of every
// member's compressions run as one batched launch (linalg.cu / mpsops.cu,
// "batched launches"), and the host waits once per SVD site for the kept
// ranks of all members instead of once per member.  Small simulations, whose
// single launches occupy a few SMs for a few microseconds, then fill the GPU
// and pay the launch and synchronisation latency once for the whole group.
//
// Every member runs the kernel variants and launch geometries of its own
// single-simulation step (vp_step), so its result does not depend on the
// group.  The method is that of vp_step: SI "Compressed time evolution
// algorithm" (RK4, level C1) with the compression of SI "Canonicalization and
// Compression" (QR sweep left to right, truncated-SVD sweep right to left,
// truncation-error equation of "MPS Representation"), the field of "Problem
// Statement" (density by SI "Integration", periodic Poisson) and the
// operator of SI "Upwind time evolution" / "Dot Product".
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "mpo_build.hpp"
#include "sim.hpp"

namespace vp {
namespace {

constexpr double kPairTolG = 1e-13;  // IG: bonds inside the (x_j, v_j) pairs (as in the single path)

// Device record of one compression problem: its status words, and the kept
// rank, truncation error and entanglement entropy of its last SVD site.
struct TaskDev {
  DevStatus st;
  int rank;
  int pad;
  double err, ent;
};

// Workspaces of one compression problem (device, grow-only).
struct Work {
  DevBuf F[2], P[2], gemm;                                       // QR sweep
  DevBuf piv, fac, p, q1, r, p2, q2, tmp, tmp2, l, j, vec, a, b, c;  // SVD site
  BScratch main, side;                                           // scratch of the batched launchers
};

void release_work(vp_ctx* ctx, Work& w) {
  for (DevBuf* b : {&w.F[0], &w.F[1], &w.P[0], &w.P[1], &w.gemm, &w.piv, &w.fac, &w.p, &w.q1, &w.r, &w.p2, &w.q2,
                    &w.tmp, &w.tmp2, &w.l, &w.j, &w.vec, &w.a, &w.b, &w.c})
    release(ctx, *b);
  release_scratch(ctx, w.main);
  release_scratch(ctx, w.side);
}

struct Member {
  vp_sim* sim = nullptr;
  Work wa, wb;          // the two compressions of a stage (wa also decomposes the field)
  DevBuf rem;           // field decomposition: the remaining reshaped vector
  DevBuf pend, dtmp, T, da, db;  // density: pending v contraction, products, expansion
  std::vector<DevBuf> xc;        // density: x cores after the v sites are absorbed
  std::vector<int> xr;
  bool have_pend = false;
  int pend_l = 1, pend_r = 1;
  std::vector<double> errs;      // per-bond truncation errors of the final compression
  int status = VP_OK;            // VP_OK, or the error that stopped this member
  const mps_t* fi = nullptr;     // stage state f_i and running sum of the current step
  const mps_t* acc = nullptr;
};

// One compression problem of a lockstep sweep.
struct Task {
  mps_t* s = nullptr;
  int chi = 1 << 30;
  double tol = 0.0;
  bool pairs = false;  // IG pair rule
  int fp32 = 0;        // FP32 contraction mode of the sweeps' GEMMs
  double* errs = nullptr;
  double* ent = nullptr;
  Work* w = nullptr;
  int slot = 0;    // TaskDev record
  int member = 0;
  int* status = nullptr;  // the owner's status (a member's, or a creation job's)
  // the SVD site in flight
  int k = 0, m = 0, c = 0, pl = 0, q = 0, p = 0, r = 1;
  bool tall = false;
};

}  // namespace
}  // namespace vp

struct vp_group {
  vp_ctx* ctx = nullptr;
  int cap = 0;
  std::vector<vp::Member*> mem;
  vp::TaskDev* d_task = nullptr;  // 2 * cap records (device)
  vp::TaskDev* h_task = nullptr;  // pinned mirror
  vp::TaskDev* h_init = nullptr;  // pinned: the records at the start of a step
  double* d_we = nullptr;         // per member: W_E, mass of f_n; then scratch for the other stages
  double* h_we = nullptr;
  cudaStream_t side = nullptr;
  cudaEvent_t ev_qf[2] = {nullptr, nullptr}, ev_qd[2] = {nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // diagnostics of the last step: host wall time, time spent waiting for the
  // device, host waits, kernel launches
  double stat_step_ms = 0, stat_wait_ms = 0;
  int64_t stat_waits = 0, stat_launches = 0;
  // batched MPS creation: workspaces and buffers of each job (grow-only)
  std::vector<vp::Work> cwork;
  std::vector<vp::DevBuf> cgrid, csites, crem;
};

namespace vp {
namespace {

using Tasks = std::vector<Task*>;

// Launches inside the scope run on the group's side stream, and buffers that
// grow there are released in that stream's order.
struct OnSide {
  vp_ctx* c;
  cudaStream_t* side;
  OnSide(vp_ctx* ctx, cudaStream_t* s) : c(ctx), side(s) { std::swap(c->stream, *side); }
  ~OnSide() { std::swap(c->stream, *side); }
};

bool alive(const vp_group*, const Task* t) { return *t->status == VP_OK; }

// Wait for the group's stream, read every problem's record, and stop the
// members whose kernels reported an error (each member fails alone).
double wall_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int sync_records(vp_group* g, int ntask_slots) {
  vp_ctx* ctx = g->ctx;
  VP_CUDA(ctx, cudaMemcpyAsync(g->h_task, g->d_task, sizeof(TaskDev) * ntask_slots, cudaMemcpyDeviceToHost,
                               ctx->stream));
  const double t0 = wall_ms();
  VP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  g->stat_wait_ms += wall_ms() - t0;
  g->stat_waits++;
  return VP_OK;
}

void mark_failures(vp_group* g, const Tasks& ts) {
  for (Task* t : ts) {
    const int e = g->h_task[t->slot].st.err;
    if (e != 0 && *t->status == VP_OK) *t->status = e == 1 ? VP_ETIMEOUT : VP_ENUMERIC;
  }
}

Tasks live(const vp_group* g, const Tasks& ts) {
  Tasks o;
  for (Task* t : ts)
    if (alive(g, t)) o.push_back(t);
  return o;
}

std::vector<int> live_ids(const vp_group* g, const std::vector<int>& ids) {
  std::vector<int> o;
  for (int i : ids)
    if (g->mem[i]->status == VP_OK) o.push_back(i);
  return o;
}

// The contraction mode of a member's GEMMs (its whole step, as in vp_step).
int fp32_of(const Member* mb) { return mb->sim->cfg.precision == VP_PREC_FP32_CONTRACT ? 1 : 0; }

// Algorithmic flops of an m x n Householder QR (the single path's count).
double qr_flops(double m, double n) {
  return m >= n ? 2 * m * n * n - 2.0 / 3.0 * n * n * n : 2 * n * m * m - 2.0 / 3.0 * m * m * m;
}

// Work of a problem's launches, added to its member's flop counters.
void account(vp_group* g, const Task* t, double qr, double formq, double gemm, double jac) {
  if (t->member < 0 || t->member >= (int)g->mem.size()) return;
  Flops& f = g->mem[t->member]->sim->flops;
  f.qr += qr;
  f.formq += formq;
  f.gemm += gemm;
  f.jacobi += jac;
}

// A batched launch bracketed for the context's kernel-class timing (the
// events go on the stream the launches go on).
template <class F>
int timed(vp_ctx* ctx, int cls, double work, F&& launch) {
  prof_begin(ctx, cls);
  const int st = launch();
  prof_end(ctx, cls, work);
  return st;
}

// Status words and rank records of every problem back to their initial
// state (counters zero, the context's wait limit), in stream order.
int reset_records(vp_group* g) {
  vp_ctx* ctx = g->ctx;
  for (int r = 0; r < 2 * g->cap; ++r) g->h_init[r].st.wait_clocks = ctx->wait_clocks;
  VP_CUDA(ctx, cudaMemcpyAsync(g->d_task, g->h_init, sizeof(TaskDev) * 2 * g->cap, cudaMemcpyHostToDevice,
                               ctx->stream));
  return VP_OK;
}

// ------------------------------------------------------------ QR sweep
// The lockstep form of api.cu's qr_sweep: at site k of every problem with a
// site k + 1, the Householder QR of the (2 r_{k-1} x r_k) reshape, R
// multiplied into core k + 1 on the group's stream, Q (the new core k)
// formed on the side stream while site k + 1 is factored.
int qr_sweep(vp_group* g, const Tasks& all) {
  vp_ctx* ctx = g->ctx;
  struct Join {
    vp_group* g;
    bool busy[2] = {false, false};
    ~Join() {
      for (int b = 0; b < 2; ++b)
        if (busy[b]) cudaStreamWaitEvent(g->ctx->stream, g->ev_qd[b], 0);
    }
  } join{g};
  int kend = 0;
  for (Task* t : all) kend = std::max(kend, t->s->n - 1);
  for (int k = 0; k < kend; ++k) {
    Tasks ts;
    for (Task* t : all)
      if (k < t->s->n - 1) ts.push_back(t);
    if (ts.empty()) continue;
    const int b = k & 1;
    if (join.busy[b]) {  // the Q formation two sites back still reads buffer b
      VP_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, g->ev_qd[b], 0));
      join.busy[b] = false;
    }
    std::vector<BColMajor> cm;
    std::vector<BQR> qr;
    std::vector<BFormQ> fq;
    std::vector<BGemm> gr;
    std::vector<int> pv;
    for (Task* t : ts) {
      mps_t* s = t->s;
      Work& w = *t->w;
      w.main.st = w.side.st = &g->d_task[t->slot].st;
      const int m = 2 * s->r[k], n = s->r[k + 1], p = std::min(m, n), nn = 2 * s->r[k + 2];
      VP_TRY(reserve(ctx, w.F[b], (size_t)m * n));
      VP_TRY(reserve(ctx, w.P[b], (size_t)2 * m + p + 8));
      VP_TRY(reserve(ctx, w.gemm, (size_t)p * nn));
      double* tau = w.P[b].p;
      cm.push_back({s->core[k].p, m, n, w.F[b].p});
      qr.push_back({w.F[b].p, m, n, tau, w.P[b].p + p + 8, &w.main});
      fq.push_back({w.F[b].p, m, n, tau, s->core[k].p, &w.side});
      gr.push_back({BG_RB, t->fp32, p, nn, n, 1.0, w.F[b].p, m, s->core[k + 1].p, nn, w.gemm.p, nn, &w.main});
      pv.push_back(p);
    }
    double wq = 0, wf = 0, wg = 0;
    for (size_t i = 0; i < ts.size(); ++i) {
      const double m = qr[i].m, n = qr[i].n, p = pv[i], nn = gr[i].N;
      const double a = qr_flops(m, n), f = 4.0 * m * p * p - 4.0 / 3.0 * p * p * p, gm = 2.0 * p * n * nn;
      account(g, ts[i], a, f, gm, 0.0);
      wq += a;
      wf += f;
      wg += gm;
    }
    VP_TRY(blaunch_to_colmajor(ctx, ctx->stream, cm));
    VP_TRY(timed(ctx, VP_K_QR, wq, [&] { return blaunch_qr_factor(ctx, ctx->stream, qr); }));
    VP_CUDA(ctx, cudaEventRecord(g->ev_qf[b], ctx->stream));
    {
      OnSide side(ctx, &g->side);
      VP_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, g->ev_qf[b], 0));
      VP_TRY(timed(ctx, VP_K_FORMQ, wf, [&] { return blaunch_qr_formq(ctx, ctx->stream, fq); }));
      VP_CUDA(ctx, cudaEventRecord(g->ev_qd[b], ctx->stream));
    }
    join.busy[b] = true;
    VP_TRY(timed(ctx, VP_K_GEMM, wg, [&] { return blaunch_gemm(ctx, ctx->stream, gr); }));
    for (size_t i = 0; i < ts.size(); ++i) {
      std::swap(ts[i]->s->core[k + 1], ts[i]->w->gemm);
      ts[i]->s->r[k + 1] = pv[i];
    }
  }
  for (int b = 0; b < 2; ++b)
    if (join.busy[b]) {
      join.busy[b] = false;
      VP_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, g->ev_qd[b], 0));
    }
  return VP_OK;
}

// ------------------------------------------------------------ SVD sweep
// The lockstep form of api.cu's svd_sweep / svd_site: problems aligned at
// their right ends; at step j every problem with a site k = n - 1 - j >= 1
// takes the preconditioned one-sided Jacobi SVD of its (r_{k-1} x 2 r_k)
// site, then one wait for all kept ranks, then the outputs.
int svd_sweep(vp_group* g, const Tasks& all) {
  vp_ctx* ctx = g->ctx;
  int jend = 0;
  for (Task* t : all) jend = std::max(jend, t->s->n - 1);
  int slots = 0;
  for (Task* t : all) slots = std::max(slots, t->slot + 1);
  for (int jstep = 0; jstep < jend; ++jstep) {
    Tasks ts;
    for (Task* t : all)
      if (t->s->n - 1 - jstep >= 1 && alive(g, t)) ts.push_back(t);
    if (ts.empty()) continue;
    std::vector<BNormOrder> no;
    std::vector<BGather> ga;
    std::vector<BQR> qr1, qr2;
    std::vector<BGetR> gr;
    std::vector<BFormQ> fq;
    std::vector<BGemm> pq;
    std::vector<BLowerUpper> lu;
    std::vector<BCopy> cp;
    std::vector<BJacobi> jc;
    std::vector<BSelect> se;
    for (Task* t : ts) {
      mps_t* s = t->s;
      Work& w = *t->w;
      const int k = s->n - 1 - jstep;
      w.main.st = w.side.st = &g->d_task[t->slot].st;
      t->k = k;
      t->m = s->r[k];
      t->c = 2 * s->r[k + 1];
      t->pl = 2 * s->r[k - 1];
      t->tall = t->m >= t->c;
      t->q = t->tall ? t->c : t->m;
      t->p = t->tall ? t->m : t->c;
      const int q = t->q, p = t->p, m = t->m, c = t->c, pl = t->pl;
      const bool inner = t->pairs && (k & 1);  // bond inside an IG pair
      const int chi = inner ? 1 << 30 : t->chi;
      const double tol = inner ? std::min(t->tol, kPairTolG) : t->tol;
      VP_TRY(reserve(ctx, w.piv, (size_t)q / 2 + 8));
      VP_TRY(reserve(ctx, w.fac, (size_t)p * q));
      VP_TRY(reserve(ctx, w.p, (size_t)2 * p + q + 8));
      VP_TRY(reserve(ctx, w.q1, (size_t)p * q));
      VP_TRY(reserve(ctx, w.r, (size_t)q * q));
      VP_TRY(reserve(ctx, w.p2, (size_t)3 * q + 8));
      VP_TRY(reserve(ctx, w.q2, (size_t)q * q));
      if (t->tall) VP_TRY(reserve(ctx, w.tmp2, (size_t)pl * q));
      VP_TRY(reserve(ctx, w.tmp, (size_t)q * q));
      if (t->tall)
        VP_TRY(reserve(ctx, w.l, (size_t)q * q));
      else
        VP_TRY(reserve(ctx, w.j, (size_t)q * q));
      VP_TRY(reserve(ctx, w.vec, (size_t)2 * q + 8));
      int* piv = (int*)w.piv.p;
      no.push_back({s->core[k].p, m, c, t->tall ? 1 : 0, piv});
      ga.push_back({s->core[k].p, m, c, piv, t->tall ? 1 : 0, w.fac.p});
      qr1.push_back({w.fac.p, p, q, w.p.p, w.p.p + q + 8, &w.main});
      gr.push_back({w.fac.p, p, q, w.r.p});
      qr2.push_back({w.r.p, q, q, w.p2.p, w.p2.p + q + 8, &w.main});
      fq.push_back({w.fac.p, p, q, w.p.p, w.q1.p, &w.side});
      fq.push_back({w.r.p, q, q, w.p2.p, w.q2.p, &w.side});
      if (t->tall)
        pq.push_back({BG_AB, t->fp32, pl, q, m, 1.0, s->core[k - 1].p, m, w.q1.p, q, w.tmp2.p, q, &w.side});
      lu.push_back({w.r.p, q, w.tmp.p});
      if (t->tall) cp.push_back({w.tmp.p, w.l.p, (size_t)q * q});
      TaskDev* rec = g->d_task + t->slot;
      jc.push_back({w.tmp.p, q, q, t->tall ? nullptr : w.j.p, &rec->st});
      int* perm = (int*)w.vec.p;
      double* sigma = w.vec.p + (q + 1) / 2 + 4;
      se.push_back({w.tmp.p, q, q, chi, tol, perm, sigma, &rec->rank, &rec->err, &rec->st});
    }
    double wq = 0, wf = 0, wp = 0;
    for (Task* t : ts) {
      const double p = t->p, q = t->q;
      const double a = qr_flops(p, q) + qr_flops(q, q), f = 4.0 * p * q * q - 4.0 / 3.0 * q * q * q + 8.0 / 3.0 * q * q * q;
      const double gm = t->tall ? 2.0 * t->pl * q * t->m : 0.0;
      account(g, t, a, f, gm, 0.0);
      wq += a;
      wf += f;
      wp += gm;
    }
    // A Pi = Q1 R1, R1^T = Q2 L^T
    VP_TRY(blaunch_norm_order(ctx, ctx->stream, no));
    VP_TRY(blaunch_gather_cm(ctx, ctx->stream, ga));
    VP_TRY(timed(ctx, VP_K_QR, wq, [&] {
      int st = blaunch_qr_factor(ctx, ctx->stream, qr1);
      if (st == VP_OK) st = blaunch_qr_getr(ctx, ctx->stream, gr);
      if (st == VP_OK) st = blaunch_qr_factor(ctx, ctx->stream, qr2);
      return st;
    }));
    // Q1, Q2 (and, tall, P Q1) on the side stream while the Jacobi SVD runs
    VP_CUDA(ctx, cudaEventRecord(g->ev_fork, ctx->stream));
    VP_CUDA(ctx, cudaStreamWaitEvent(g->side, g->ev_fork, 0));
    {
      OnSide side(ctx, &g->side);
      VP_TRY(timed(ctx, VP_K_FORMQ, wf, [&] { return blaunch_qr_formq(ctx, ctx->stream, fq); }));
      VP_TRY(timed(ctx, VP_K_GEMM, wp, [&] { return blaunch_gemm(ctx, ctx->stream, pq); }));
      VP_CUDA(ctx, cudaEventRecord(g->ev_join, ctx->stream));
    }
    struct SideJoin {
      vp_group* g;
      ~SideJoin() { cudaStreamWaitEvent(g->ctx->stream, g->ev_join, 0); }
    } side_join{g};
    VP_TRY(blaunch_lower_from_upper(ctx, ctx->stream, lu));
    VP_TRY(blaunch_copy(ctx, ctx->stream, cp));
    const size_t jac_mark = ctx->prof_on ? ctx->prof_marks.size() : (size_t)-1;
    VP_TRY(timed(ctx, VP_K_JACOBI, 0.0, [&] { return blaunch_jacobi(ctx, ctx->stream, jc); }));
    VP_TRY(timed(ctx, VP_K_SELECT, 0.0, [&] { return blaunch_select(ctx, ctx->stream, se); }));
    // one wait for the kept ranks of every problem at this step
    VP_TRY(sync_records(g, slots));
    mark_failures(g, ts);
    {  // Jacobi work from the sweeps each problem took (the single path's count)
      double wj = 0.0;
      for (Task* t : ts) {
        const double q = t->q, sweeps = g->h_task[t->slot].st.pad2;
        const double j = q > 1 ? sweeps * 0.5 * q * (q - 1) * (6.0 * q + (t->tall ? 0.0 : 4.0 * q)) : 0.0;
        account(g, t, 0, 0, 0, j);
        wj += j;
      }
      if (ctx->prof_on) ctx->prof_work[VP_K_JACOBI] += wj;
      if (jac_mark != (size_t)-1 && jac_mark < ctx->prof_marks.size()) ctx->prof_marks[jac_mark].m = (int)ts.size();
    }
    ts = live(g, ts);
    std::vector<BSvdOut> so;
    std::vector<BSvdOutWide> sw;
    std::vector<BGemm> g2, g3, g5;
    std::vector<BScatter> sc;
    for (Task* t : ts) {
      mps_t* s = t->s;
      Work& w = *t->w;
      const TaskDev& rec = g->h_task[t->slot];
      const int r = rec.rank, k = t->k, q = t->q, m = t->m, c = t->c, pl = t->pl;
      t->r = r;
      if (t->errs) t->errs[k - 1] = rec.err;
      if (t->ent) t->ent[k - 1] = rec.ent;
      VP_TRY(reserve(ctx, w.a, (size_t)r * q + 8));
      VP_TRY(reserve(ctx, w.b, (size_t)q * r + 8));
      int* perm = (int*)w.vec.p;
      double* sigma = w.vec.p + (q + 1) / 2 + 4;
      const int* piv = (const int*)w.piv.p;
      if (t->tall) {
        // core_{k-1} <- (P Q1) (U_L S), U_L S = L V_L; core_k <- scatter(V_L^T Q2^T)
        VP_TRY(reserve(ctx, w.gemm, (size_t)pl * r));
        VP_TRY(reserve(ctx, w.c, (size_t)r * q));
        VP_TRY(reserve(ctx, s->core[k], (size_t)r * c));
        so.push_back({w.tmp.p, nullptr, q, q, r, perm, sigma, w.a.p, nullptr});
        g2.push_back({BG_ABT, t->fp32, q, r, q, 1.0, w.l.p, q, w.a.p, q, w.b.p, r, &w.main});
        g2.push_back({BG_ABT, t->fp32, r, q, q, 1.0, w.a.p, q, w.q2.p, q, w.c.p, q, &w.main});
        g3.push_back({BG_AB, t->fp32, pl, r, q, 1.0, w.tmp2.p, q, w.b.p, r, w.gemm.p, r, &w.main});
        sc.push_back({w.c.p, r, q, piv, 1, s->core[k].p});
      } else {
        // core_k <- U_L^T Q1^T; core_{k-1} <- P Pi (Q2 V_L S)
        VP_TRY(reserve(ctx, s->core[k], (size_t)r * c));
        VP_TRY(reserve(ctx, w.c, (size_t)m * r));
        VP_TRY(reserve(ctx, w.tmp2, (size_t)m * r));
        VP_TRY(reserve(ctx, w.gemm, (size_t)pl * r));
        sw.push_back({w.tmp.p, w.j.p, q, r, perm, w.a.p, w.b.p});
        g2.push_back({BG_ABT, t->fp32, r, c, m, 1.0, w.a.p, m, w.q1.p, m, s->core[k].p, c, &w.main});
        g3.push_back({BG_AB, t->fp32, m, r, m, 1.0, w.q2.p, m, w.b.p, r, w.c.p, r, &w.main});
        sc.push_back({w.c.p, m, r, piv, 0, w.tmp2.p});
        g5.push_back({BG_AB, t->fp32, pl, r, m, 1.0, s->core[k - 1].p, m, w.tmp2.p, r, w.gemm.p, r, &w.main});
      }
    }
    double wo = 0.0;
    for (const auto* v : {&g2, &g3, &g5})
      for (const BGemm& x : *v) wo += 2.0 * x.M * x.N * x.K;
    for (Task* t : ts) {
      const double q = t->q, r = t->r, m = t->m, c = t->c, pl = t->pl;
      account(g, t, 0, 0, t->tall ? 2.0 * pl * r * q + 4.0 * r * q * q : 2.0 * r * c * m + 2.0 * m * r * m + 2.0 * pl * r * m,
              0);
    }
    VP_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, g->ev_join, 0));
    VP_TRY(timed(ctx, VP_K_GEMM, wo, [&] {
      int st = blaunch_svd_outputs(ctx, ctx->stream, so);
      if (st == VP_OK) st = blaunch_svd_outputs_wide(ctx, ctx->stream, sw);
      if (st == VP_OK) st = blaunch_gemm(ctx, ctx->stream, g2);
      if (st == VP_OK) st = blaunch_gemm(ctx, ctx->stream, g3);
      if (st == VP_OK) st = blaunch_scatter(ctx, ctx->stream, sc);
      if (st == VP_OK) st = blaunch_gemm(ctx, ctx->stream, g5);
      return st;
    }));
    for (Task* t : ts) {
      std::swap(t->s->core[t->k - 1], t->w->gemm);
      t->s->r[t->k] = t->r;
    }
  }
  return VP_OK;
}

int compress(vp_group* g, const Tasks& ts) {
  VP_TRY(qr_sweep(g, ts));
  return svd_sweep(g, ts);
}

// ------------------------------------------------------------ decomposition
// A site-ordered device vector (2^n) as an MPS, for several problems at once:
// api.cu's from_vector -- a chain of Householder QR factorisations of the
// reshapes (MPS decomposition, "MPS Representation"), then the truncated-SVD
// sweep -- in lockstep over the sites.
struct VecJob {
  mps_t* out;
  const double* vec;  // device, 2^n, read before anything is written
  int n;
  int chi;
  double tol;
  bool pairs;  // IG pair rule in the SVD sweep
  int fp32;
  Work* w;
  DevBuf* rem;  // the remaining reshaped vector (2^n)
  int slot;
  int* status;
};

int from_vectors(vp_group* g, const std::vector<VecJob>& jobs) {
  vp_ctx* ctx = g->ctx;
  std::vector<BCopy> cp;
  int nmax = 0;
  for (const VecJob& jb : jobs) {
    const size_t N = (size_t)1 << jb.n;
    if (jb.out->n != jb.n || jb.out->ctx != ctx) {
      mps_free(jb.out);
      mps_init(ctx, jb.out, jb.n);
    } else {
      jb.out->r.assign(jb.n + 1, 1);  // the cores' buffers are kept and overwritten
    }
    jb.w->main.st = jb.w->side.st = &g->d_task[jb.slot].st;
    VP_TRY(reserve(ctx, *jb.rem, N));
    cp.push_back({jb.vec, jb.rem->p, N});
    nmax = std::max(nmax, jb.n);
  }
  VP_TRY(blaunch_copy(ctx, ctx->stream, cp));
  std::vector<int> rr(jobs.size(), 1);
  for (int k = 0; k + 1 < nmax; ++k) {
    std::vector<BColMajor> cm;
    std::vector<BQR> qr;
    std::vector<BFormQ> fq;
    std::vector<BGetR> gr;
    for (size_t a = 0; a < jobs.size(); ++a) {
      const VecJob& jb = jobs[a];
      if (k + 1 >= jb.n) continue;
      Work& w = *jb.w;
      const size_t N = (size_t)1 << jb.n;
      const int m = 2 * rr[a];
      const size_t cols = N >> (k + 1);
      if (cols > (size_t)1 << 30) return fail(ctx, VP_ECAPACITY, "vector too long");
      const int nc = (int)cols, p = std::min(m, nc);
      VP_TRY(reserve(ctx, w.fac, (size_t)m * nc));
      VP_TRY(reserve(ctx, w.p, (size_t)2 * m + p + 8));
      VP_TRY(reserve(ctx, jb.out->core[k], (size_t)m * p));
      cm.push_back({jb.rem->p, m, nc, w.fac.p});
      qr.push_back({w.fac.p, m, nc, w.p.p, w.p.p + p + 8, &w.main});
      fq.push_back({w.fac.p, m, nc, w.p.p, jb.out->core[k].p, &w.main});
      gr.push_back({w.fac.p, m, nc, jb.rem->p});
      jb.out->r[k + 1] = p;
      rr[a] = p;
    }
    VP_TRY(blaunch_to_colmajor(ctx, ctx->stream, cm));
    VP_TRY(blaunch_qr_factor(ctx, ctx->stream, qr));
    VP_TRY(blaunch_qr_formq(ctx, ctx->stream, fq));
    VP_TRY(blaunch_qr_getr(ctx, ctx->stream, gr));
  }
  cp.clear();
  std::vector<Task> tasks(jobs.size());
  Tasks ts;
  for (size_t a = 0; a < jobs.size(); ++a) {
    const VecJob& jb = jobs[a];
    VP_TRY(reserve(ctx, jb.out->core[jb.n - 1], (size_t)2 * rr[a]));
    cp.push_back({jb.rem->p, jb.out->core[jb.n - 1].p, (size_t)2 * rr[a]});
    Task& t = tasks[a];
    t.s = jb.out;
    t.chi = jb.chi;
    t.tol = jb.tol;
    t.pairs = jb.pairs;
    t.fp32 = jb.fp32;
    t.w = jb.w;
    t.slot = jb.slot;
    t.status = jb.status;
    if (jb.n > 1) ts.push_back(&t);
  }
  VP_TRY(blaunch_copy(ctx, ctx->stream, cp));
  return svd_sweep(g, ts);
}

// E (device, 2^nx) of every member as an MPS in the site order of the x
// bits, truncated at e_tol and capped at e_chi (the field MPS holds x bits
// only: no pair rule).
int field_mps(vp_group* g, const std::vector<int>& ids) {
  vp_ctx* ctx = g->ctx;
  std::vector<BPermute> pm;
  std::vector<VecJob> jobs;
  for (int i : ids) {
    Member* mb = g->mem[i];
    vp_sim* s = mb->sim;
    const int nx = s->lay.nx;
    const double* ev = s->E.p;
    if (xdesc(&s->lay)) {
      VP_TRY(reserve(ctx, s->evec, (size_t)1 << nx));
      pm.push_back({s->E.p, nx, 0, VP_SEQ_S2, s->evec.p, 0});
      ev = s->evec.p;
    }
    jobs.push_back({&s->em, ev, nx, s->cfg.e_chi > 0 ? s->cfg.e_chi : 1 << 30, s->cfg.e_tol, false, fp32_of(mb),
                    &mb->wa, &mb->rem, 2 * i, &mb->status});
  }
  VP_TRY(blaunch_permute(ctx, ctx->stream, pm));
  return from_vectors(g, jobs);
}

// L(E) = U + diag(E) (x) D_v of every member (api.cu's assemble_operator):
// all sites of all members in one batched launch.
int assemble(vp_group* g, const std::vector<int>& ids) {
  vp_ctx* ctx = g->ctx;
  std::vector<BAssemble> as;
  for (int i : ids) {
    vp_sim* s = g->mem[i]->sim;
    const int n = (int)s->dims.size();
    const mps_t& em = s->em;
    std::vector<int> tw(n + 1), w(n + 1);
    int px = 0, pv = 0;
    tw[0] = 1;
    for (int k = 0; k < n; ++k) {
      if (s->dims[k] == 0) ++px; else ++pv;
      tw[k + 1] = em.r[px] * s->Dv.w[pv];
    }
    w[0] = w[n] = 1;
    for (int k = 1; k < n; ++k) w[k] = s->U.w[k] + tw[k];
    mpo_t& L = s->L;
    L.ctx = ctx;
    L.n = n;
    L.w = w;
    if ((int)L.core.size() != n) L.core.assign(n, DevBuf{});
    px = pv = 0;
    for (int k = 0; k < n; ++k) {
      ETermSite e{};
      if (s->dims[k] == 0) {
        e.is_x = 1;
        e.Ecore = em.core[px].p;
        e.el = em.r[px];
        e.er = em.r[px + 1];
        e.dw = s->Dv.w[pv];
        ++px;
      } else {
        e.is_x = 0;
        e.Dcore = s->Dvd[pv].p;
        e.dl = s->Dv.w[pv];
        e.dr = s->Dv.w[pv + 1];
        e.ew = em.r[px];
        ++pv;
      }
      VP_TRY(reserve(ctx, L.core[k], (size_t)w[k] * 4 * w[k + 1]));
      as.push_back({s->Ud[k].p, s->U.w[k], s->U.w[k + 1], e, k == 0, k == n - 1, L.core[k].p, w[k], w[k + 1]});
    }
  }
  return blaunch_assemble(ctx, ctx->stream, as);
}

// rho = dv * (every v site contracted with [1, 1], the x chain expanded) for
// every member (api.cu's density), lockstep over the site index.
int density(vp_group* g, const std::vector<int>& ids, const std::vector<const mps_t*>& fs) {
  vp_ctx* ctx = g->ctx;
  int nmax = 0;
  for (size_t a = 0; a < ids.size(); ++a) {
    Member* mb = g->mem[ids[a]];
    mb->have_pend = false;
    mb->pend_l = mb->pend_r = 1;
    mb->xr.assign(1, 1);
    if (mb->xc.size() < (size_t)mb->sim->lay.nx) mb->xc.resize(mb->sim->lay.nx);
    nmax = std::max(nmax, fs[a]->n);
  }
  std::vector<int> nxc(ids.size(), 0);  // x cores filled so far
  for (int k = 0; k < nmax; ++k) {
    std::vector<BPhysSum> ph;
    std::vector<BGemm> gm;
    std::vector<BCopy> cp;
    std::vector<int> vsite, vgemm;
    for (size_t a = 0; a < ids.size(); ++a) {
      Member* mb = g->mem[ids[a]];
      const mps_t* f = fs[a];
      if (k >= f->n || mb->sim->dims[k] != 1) continue;
      const int rl = f->r[k], rr = f->r[k + 1];
      VP_TRY(reserve(ctx, mb->T, (size_t)rl * rr));
      ph.push_back({f->core[k].p, rl, rr, mb->T.p});
      vsite.push_back((int)a);
    }
    VP_TRY(blaunch_phys_sum(ctx, ctx->stream, ph));
    for (int a : vsite) {
      Member* mb = g->mem[ids[a]];
      const mps_t* f = fs[a];
      const int rl = f->r[k], rr = f->r[k + 1];
      if (!mb->have_pend) {
        std::swap(mb->pend, mb->T);
        mb->pend_l = rl;
        mb->pend_r = rr;
        mb->have_pend = true;
      } else {
        VP_TRY(reserve(ctx, mb->dtmp, (size_t)mb->pend_l * rr));
        gm.push_back({BG_AB, fp32_of(mb), mb->pend_l, rr, rl, 1.0, mb->pend.p, rl, mb->T.p, rr, mb->dtmp.p, rr,
                      &mb->wa.main});
        vgemm.push_back(a);
      }
    }
    for (size_t a = 0; a < ids.size(); ++a) {
      Member* mb = g->mem[ids[a]];
      const mps_t* f = fs[a];
      if (k >= f->n || mb->sim->dims[k] != 0) continue;
      const int rl = f->r[k], rr = f->r[k + 1];
      DevBuf& c = mb->xc[nxc[a]++];
      if (mb->have_pend) {
        VP_TRY(reserve(ctx, c, (size_t)mb->pend_l * 2 * rr));
        gm.push_back({BG_AB, fp32_of(mb), mb->pend_l, 2 * rr, rl, 1.0, mb->pend.p, rl, f->core[k].p, 2 * rr, c.p, 2 * rr,
                      &mb->wa.main});
        mb->have_pend = false;
        mb->xr.back() = mb->pend_l;
      } else {
        VP_TRY(reserve(ctx, c, (size_t)rl * 2 * rr));
        cp.push_back({f->core[k].p, c.p, (size_t)rl * 2 * rr});
      }
      mb->xr.push_back(rr);
    }
    VP_TRY(blaunch_gemm(ctx, ctx->stream, gm));
    VP_TRY(blaunch_copy(ctx, ctx->stream, cp));
    for (int a : vgemm) {
      Member* mb = g->mem[ids[a]];
      std::swap(mb->pend, mb->dtmp);
      mb->pend_r = fs[a]->r[k + 1];
    }
  }
  // trailing v sites: absorbed into the last x core on its right
  {
    std::vector<BGemm> gm;
    std::vector<int> tr;
    for (size_t a = 0; a < ids.size(); ++a) {
      Member* mb = g->mem[ids[a]];
      if (!mb->have_pend) continue;
      DevBuf& last = mb->xc[nxc[a] - 1];
      const int lx = mb->xr[mb->xr.size() - 2], rx = mb->xr.back();
      VP_TRY(reserve(ctx, mb->dtmp, (size_t)lx * 2 * mb->pend_r));
      gm.push_back({BG_AB, fp32_of(mb), lx * 2, mb->pend_r, rx, 1.0, last.p, rx, mb->pend.p, mb->pend_r, mb->dtmp.p,
                    mb->pend_r, &mb->wa.main});
      tr.push_back((int)a);
    }
    VP_TRY(blaunch_gemm(ctx, ctx->stream, gm));
    for (int a : tr) {
      Member* mb = g->mem[ids[a]];
      std::swap(mb->xc[nxc[a] - 1], mb->dtmp);
      mb->xr.back() = mb->pend_r;
    }
  }
  // expand the x chain (api.cu's to_dense_dev), then rho = dv * (permuted) dense
  int xmax = 0;
  std::vector<BCopy> cp;
  std::vector<size_t> rows(ids.size(), 2);
  for (size_t a = 0; a < ids.size(); ++a) {
    Member* mb = g->mem[ids[a]];
    const size_t e0 = (size_t)mb->xr[0] * 2 * mb->xr[1];
    VP_TRY(reserve(ctx, mb->da, e0));
    cp.push_back({mb->xc[0].p, mb->da.p, e0});
    xmax = std::max(xmax, nxc[a]);
  }
  VP_TRY(blaunch_copy(ctx, ctx->stream, cp));
  for (int k = 1; k < xmax; ++k) {
    std::vector<BGemm> gm;
    std::vector<int> us;
    for (size_t a = 0; a < ids.size(); ++a) {
      Member* mb = g->mem[ids[a]];
      if (k >= nxc[a]) continue;
      const int rk = mb->xr[k], rn = mb->xr[k + 1];
      if (rows[a] > (size_t)1 << 26) return fail(ctx, VP_ECAPACITY, "density: too many sites");
      VP_TRY(reserve(ctx, mb->db, rows[a] * 2 * rn));
      gm.push_back({BG_AB, fp32_of(mb), (int)rows[a], 2 * rn, rk, 1.0, mb->da.p, rk, mb->xc[k].p, 2 * rn, mb->db.p, 2 * rn,
                    &mb->wa.main});
      us.push_back((int)a);
    }
    VP_TRY(blaunch_gemm(ctx, ctx->stream, gm));
    for (int a : us) {
      Member* mb = g->mem[ids[a]];
      std::swap(mb->da, mb->db);
      rows[a] *= 2;
    }
  }
  std::vector<BPermute> pm;
  std::vector<BScale> sc;
  cp.clear();
  for (size_t a = 0; a < ids.size(); ++a) {
    Member* mb = g->mem[ids[a]];
    vp_sim* s = mb->sim;
    const size_t Nx = (size_t)1 << s->lay.nx;
    if (xdesc(&s->lay))  // the expansion is indexed by the x bits in site order: undo the bit reversal
      pm.push_back({mb->da.p, s->lay.nx, 0, VP_SEQ_S2, s->rho.p, 1});
    else
      cp.push_back({mb->da.p, s->rho.p, Nx});
    sc.push_back({s->rho.p, Nx, grid_dv(&s->lay)});
  }
  VP_TRY(blaunch_permute(ctx, ctx->stream, pm));
  VP_TRY(blaunch_copy(ctx, ctx->stream, cp));
  return blaunch_scale(ctx, ctx->stream, sc);
}

// Field of a stage for every member: rho -> E (W_E and mass of f_n at
// stage 0) -> E as an MPS -> L(E).
int stage_operator(vp_group* g, const std::vector<int>& ids, const std::vector<const mps_t*>& fs, int stage) {
  VP_TRY(density(g, ids, fs));
  std::vector<BPoisson> po;
  for (int i : ids) {
    vp_sim* s = g->mem[i]->sim;
    double* we = g->d_we + 2 * (stage == 0 ? i : g->cap + i);
    po.push_back({s->rho.p, 1 << s->lay.nx, grid_dx(&s->lay), s->E.p, we});
  }
  VP_TRY(blaunch_poisson(g->ctx, g->ctx->stream, po));
  VP_TRY(field_mps(g, ids));
  return assemble(g, live_ids(g, ids));
}

// out_m = alpha a_m + beta (L_m b_m) for every member (api.cu's site_sum_mps):
// all sites of all members in one batched launch.
struct SumSpec {
  double alpha;
  const mps_t* a;
  double beta;
  const mpo_t* B;
  const mps_t* b;
  mps_t* out;
};
int site_sums(vp_ctx* ctx, const std::vector<SumSpec>& v) {
  std::vector<BSiteSum> ss;
  for (const SumSpec& sp : v) {
    const int n = sp.b->n;
    std::vector<int> r(n + 1, 1);
    for (int k = 1; k < n; ++k) r[k] = (sp.a ? sp.a->r[k] : 0) + sp.b->r[k] * (sp.B ? sp.B->w[k] : 1);
    if (sp.out->n != n) {
      mps_free(sp.out);
      mps_init(ctx, sp.out, n);
    }
    for (int k = 0; k < n; ++k) {
      SiteSum s{};
      s.a = sp.a ? sp.a->core[k].p : nullptr;
      s.al = sp.a ? sp.a->r[k] : 0;
      s.ar = sp.a ? sp.a->r[k + 1] : 0;
      s.b = sp.b->core[k].p;
      s.bl = sp.b->r[k];
      s.br = sp.b->r[k + 1];
      s.B = sp.B ? sp.B->core[k].p : nullptr;
      s.wl = sp.B ? sp.B->w[k] : 1;
      s.wr = sp.B ? sp.B->w[k + 1] : 1;
      s.alpha = (k == 0) ? sp.alpha : 1.0;
      s.beta = (k == 0) ? sp.beta : 1.0;
      s.first = (k == 0);
      s.last = (k == n - 1);
      VP_TRY(reserve(ctx, sp.out->core[k], (size_t)r[k] * 2 * r[k + 1]));
      ss.push_back({s, sp.out->core[k].p, r[k], r[k + 1]});
    }
    sp.out->r = r;
  }
  double bytes = 0.0;
  for (const BSiteSum& b : ss)
    bytes += 8.0 * ((double)b.ol * 2 * b.orr + (b.s.a ? (double)b.s.al * 2 * b.s.ar : 0.0) +
                    (double)b.s.bl * 2 * b.s.br + (b.s.B ? (double)b.s.wl * 4 * b.s.wr : 0.0));
  return timed(ctx, VP_K_APPLY, bytes, [&] { return blaunch_site_sum(ctx, ctx->stream, ss); });
}

// One RK4-C1 step of every live member (api.cu's sim_step_impl / c1_stage).
int group_step(vp_group* g, vp_record* recs) {
  vp_ctx* ctx = g->ctx;
  static const double A[3] = {0.5, 0.5, 1.0};
  static const double B[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  const int nm = (int)g->mem.size();
  std::vector<int> ids;
  for (int i = 0; i < nm; ++i)
    if (g->mem[i]->status == VP_OK) ids.push_back(i);
  if (ids.empty()) return VP_OK;
  VP_TRY(reset_records(g));
  for (int i : ids) {
    Member* mb = g->mem[i];
    mb->fi = mb->acc = &mb->sim->f;
    mb->errs.assign(std::max(1, mb->sim->f.n), 0.0);
  }
  for (int st = 0; st < 4; ++st) {
    ids = live_ids(g, ids);
    if (ids.empty()) break;
    std::vector<const mps_t*> fs;
    for (int i : ids) fs.push_back(g->mem[i]->fi);
    VP_TRY(stage_operator(g, ids, fs, st));
    ids = live_ids(g, ids);
    std::vector<SumSpec> sums;
    std::vector<Task> tasks(2 * ids.size());
    Tasks ts;
    for (size_t a = 0; a < ids.size(); ++a) {
      const int i = ids[a];
      Member* mb = g->mem[i];
      vp_sim* s = mb->sim;
      const double dt = s->cfg.dt;
      Task& ta = tasks[2 * a];
      ta.member = i;
      ta.status = &mb->status;
      ta.slot = 2 * i;
      ta.tol = s->cfg.tol;
      ta.pairs = grouped(&s->lay);
      ta.fp32 = s->cfg.precision == VP_PREC_FP32_CONTRACT;
      ta.w = &mb->wa;
      if (st < 3) {
        sums.push_back({1.0, mb->acc, B[st] * dt, &s->L, mb->fi, &s->wa});
        sums.push_back({1.0, &s->f, A[st] * dt, &s->L, mb->fi, &s->wb});
        ta.s = &s->wa;
        Task& tb = tasks[2 * a + 1];
        tb = ta;
        tb.slot = 2 * i + 1;
        tb.s = &s->wb;
        tb.w = &mb->wb;
        ts.push_back(&ta);
        ts.push_back(&tb);
      } else {
        sums.push_back({1.0, mb->acc, B[3] * dt, &s->L, mb->fi, &s->wa});
        s->entropy.assign(std::max(1, s->f.n - 1), 0.0);
        ta.s = &s->wa;
        ta.chi = s->cfg.chi;
        ta.errs = mb->errs.data();
        ta.ent = s->entropy.data();
        ts.push_back(&ta);
      }
    }
    VP_TRY(site_sums(ctx, sums));
    VP_TRY(compress(g, ts));
    for (int i : live_ids(g, ids)) {
      Member* mb = g->mem[i];
      vp_sim* s = mb->sim;
      if (st < 3) {
        std::swap(s->acc, s->wa);
        std::swap(s->fi, s->wb);
        mb->acc = &s->acc;
        mb->fi = &s->fi;
      } else {
        std::swap(s->f, s->wa);
      }
    }
  }
  // records: one wait for every member's field energy and mass
  VP_CUDA(ctx, cudaMemcpyAsync(g->h_we, g->d_we, sizeof(double) * 2 * nm, cudaMemcpyDeviceToHost, ctx->stream));
  int slots = 2 * nm;
  VP_TRY(sync_records(g, slots));
  std::vector<Task> chk(2 * nm);
  Tasks all;
  for (int i : live_ids(g, ids))
    for (int h = 0; h < 2; ++h) {
      chk[2 * i + h].member = i;
      chk[2 * i + h].status = &g->mem[i]->status;
      chk[2 * i + h].slot = 2 * i + h;
      all.push_back(&chk[2 * i + h]);
    }
  mark_failures(g, all);
  for (int i = 0; i < nm; ++i) {
    Member* mb = g->mem[i];
    if (mb->status != VP_OK) continue;
    vp_sim* s = mb->sim;
    const double we = g->h_we[2 * i], mass = g->h_we[2 * i + 1];
    if (!std::isfinite(we)) {
      mb->status = VP_ENUMERIC;
      continue;
    }
    if (recs) {
      vp_record& rc = recs[i];
      rc.t = s->t;
      rc.field_energy = we;
      rc.mass = mass;
      rc.max_bond = *std::max_element(s->f.r.begin(), s->f.r.end());
      rc.trunc_err = mb->errs.empty() ? 0.0 : *std::max_element(mb->errs.begin(), mb->errs.end());
    }
    s->t += s->cfg.dt;
  }
  return VP_OK;
}

}  // namespace
}  // namespace vp

using namespace vp;

bool vp::lockstep_eligible(const vp_sim* s) {
  const vp_config& c = s->cfg;
  return c.level <= 1 && c.compression == VP_COMPRESS_SWEEPS && c.e_chi >= 0 &&
         (c.precision == VP_PREC_FP64 || c.precision == VP_PREC_FP32_CONTRACT) && c.tol >= 1e-13 &&
         c.e_tol >= 1e-13 && s->ecoef == 1.0;
}

extern "C" {

int vp_group_create(vp_ctx* ctx, int max_members, vp_group** out) {
  if (!ctx || !out || max_members < 1 || max_members > 4096) return fail(ctx, VP_EINVAL, "vp_group_create: bad argument");
  *out = nullptr;
  vp_group* g = new (std::nothrow) vp_group();
  if (!g) return fail(ctx, VP_ENOMEM, "vp_group_create: out of host memory");
  g->ctx = ctx;
  g->cap = max_members;
  const size_t nrec = 2 * (size_t)max_members;
  int st = VP_OK;
  g->d_task = (TaskDev*)dev_alloc(ctx, sizeof(TaskDev) * nrec);
  g->d_we = (double*)dev_alloc(ctx, sizeof(double) * 4 * max_members);
  if (!g->d_task || !g->d_we) st = fail(ctx, VP_ENOMEM, "vp_group_create: device allocation failed");
  if (st == VP_OK && (cudaMallocHost(&g->h_task, sizeof(TaskDev) * nrec) != cudaSuccess ||
                      cudaMallocHost(&g->h_init, sizeof(TaskDev) * nrec) != cudaSuccess ||
                      cudaMallocHost(&g->h_we, sizeof(double) * 4 * max_members) != cudaSuccess))
    st = fail(ctx, VP_ENOMEM, "vp_group_create: pinned allocation failed");
  if (st == VP_OK) {
    std::memset(g->h_init, 0, sizeof(TaskDev) * nrec);
    for (size_t i = 0; i < nrec; ++i) g->h_init[i].st.wait_clocks = ctx->wait_clocks;
    if (cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking) != cudaSuccess)
      st = fail(ctx, VP_ECUDA, "vp_group_create: stream creation failed");
    for (cudaEvent_t* e : {&g->ev_qf[0], &g->ev_qf[1], &g->ev_qd[0], &g->ev_qd[1], &g->ev_fork, &g->ev_join})
      if (st == VP_OK && cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess)
        st = fail(ctx, VP_ECUDA, "vp_group_create: event creation failed");
  }
  if (st == VP_OK && cudaMemsetAsync(g->d_we, 0, sizeof(double) * 4 * max_members, ctx->stream) != cudaSuccess)
    st = fail(ctx, VP_ECUDA, "vp_group_create: memset failed");
  if (st != VP_OK) {
    vp_group_destroy(g);
    return st;
  }
  *out = g;
  return VP_OK;
}

int vp_group_add(vp_group* g, vp_sim* s) {
  if (!g || !s) return VP_EINVAL;
  vp_ctx* ctx = g->ctx;
  if ((int)g->mem.size() >= g->cap) return fail(ctx, VP_ECAPACITY, "vp_group_add: the group is full");
  for (Member* m : g->mem)
    if (m->sim == s) return fail(ctx, VP_EINVAL, "vp_group_add: already a member");
  if (s->ctx != ctx || s->ctxB) return fail(ctx, VP_EINVAL, "vp_group_add: the sim must be on the group's context, one stream");
  if (!lockstep_eligible(s))
    return fail(ctx, VP_EINVAL,
                "vp_group_add: groups step level C1 with the plain sweeps, FP64 or FP32 contractions and tol >= 1e-13");
  Member* m = new (std::nothrow) Member();
  if (!m) return fail(ctx, VP_ENOMEM, "vp_group_add: out of host memory");
  m->sim = s;
  g->mem.push_back(m);
  return VP_OK;
}

static void free_member(vp_ctx* ctx, Member* m) {
  release_work(ctx, m->wa);
  release_work(ctx, m->wb);
  for (DevBuf* b : {&m->rem, &m->pend, &m->dtmp, &m->T, &m->da, &m->db}) release(ctx, *b);
  for (DevBuf& b : m->xc) release(ctx, b);
  delete m;
}

int vp_group_remove(vp_group* g, vp_sim* s) {
  if (!g || !s) return VP_EINVAL;
  for (size_t i = 0; i < g->mem.size(); ++i)
    if (g->mem[i]->sim == s) {
      free_member(g->ctx, g->mem[i]);
      g->mem.erase(g->mem.begin() + i);
      return VP_OK;
    }
  return fail(g->ctx, VP_EINVAL, "vp_group_remove: not a member");
}

int vp_group_size(const vp_group* g) { return g ? (int)g->mem.size() : -1; }

int vp_group_step(vp_group* g, vp_record* records, int* status) {
  if (!g) return VP_EINVAL;
  g->stat_wait_ms = 0;
  g->stat_waits = 0;
  const int64_t l0 = g->ctx->launches;
  const double t0 = wall_ms();
  const int st = group_step(g, records);
  g->stat_step_ms = wall_ms() - t0;
  g->stat_launches = g->ctx->launches - l0;
  if (st != VP_OK) {
    // an error of the group's own launches (not of one member's arithmetic):
    // every member that was still running is stopped with it
    cudaStreamSynchronize(g->side);
    cudaStreamSynchronize(g->ctx->stream);
    for (Member* m : g->mem)
      if (m->status == VP_OK) m->status = st;
  }
  if (status)
    for (size_t i = 0; i < g->mem.size(); ++i) status[i] = g->mem[i]->status;
  return st;
}

int vp_group_mps_create(vp_group* g, int count, const vp_layout* layouts, const double* const* f_host,
                        const int* chi, const double* tol, mps_t** out, int* status) {
  if (!g || count < 0 || (count > 0 && (!layouts || !f_host || !chi || !tol || !out || !status)))
    return VP_EINVAL;
  vp_ctx* ctx = g->ctx;
  if (count > 2 * g->cap) return fail(ctx, VP_ECAPACITY, "vp_group_mps_create: more than 2 max_members grids");
  if ((int)g->cwork.size() < count) {
    g->cwork.resize(count);
    g->cgrid.resize(count);
    g->csites.resize(count);
    g->crem.resize(count);
  }
  VP_TRY(reset_records(g));
  std::vector<BPermute> pm;
  std::vector<VecJob> jobs;
  for (int i = 0; i < count; ++i) {
    out[i] = nullptr;
    status[i] = VP_OK;
    const vp_layout* L = &layouts[i];
    if (!layout_ok(L) || !f_host[i] || chi[i] < 1 || !(tol[i] >= 1e-13)) {
      status[i] = VP_EINVAL;
      continue;
    }
    const int n = L->nx + L->nv;
    const size_t N = (size_t)1 << n;
    mps_t* m = new (std::nothrow) mps_t();
    if (!m) {
      status[i] = VP_ENOMEM;
      continue;
    }
    int st = reserve(ctx, g->cgrid[i], N);
    if (st == VP_OK) st = reserve(ctx, g->csites[i], N);
    if (st == VP_OK && cudaMemcpyAsync(g->cgrid[i].p, f_host[i], N * sizeof(double), cudaMemcpyHostToDevice,
                                       ctx->stream) != cudaSuccess)
      st = fail(ctx, VP_ECUDA, "vp_group_mps_create: copy failed");
    if (st != VP_OK) {
      delete m;
      status[i] = st;
      continue;
    }
    out[i] = m;
    pm.push_back({g->cgrid[i].p, L->nx, L->nv, L->mapping, g->csites[i].p, 0});
    jobs.push_back({m, g->csites[i].p, n, chi[i], tol[i], grouped(L), 0, &g->cwork[i], &g->crem[i], i, &status[i]});
  }
  std::vector<BCheck> ck;
  for (const VecJob& jb : jobs) ck.push_back({g->cgrid[jb.slot].p, (size_t)1 << jb.n, &g->d_task[jb.slot].st});
  int st = blaunch_check_finite(ctx, ctx->stream, ck);
  if (st == VP_OK) st = blaunch_permute(ctx, ctx->stream, pm);
  if (st == VP_OK) st = from_vectors(g, jobs);
  if (st == VP_OK) st = sync_records(g, count);
  if (st == VP_OK) {
    Tasks all;
    std::vector<Task> chk(jobs.size());
    for (size_t a = 0; a < jobs.size(); ++a) {
      chk[a].slot = jobs[a].slot;
      chk[a].status = jobs[a].status;
      all.push_back(&chk[a]);
    }
    mark_failures(g, all);
  }
  for (int i = 0; i < count; ++i)
    if (out[i] && (st != VP_OK || status[i] != VP_OK)) {
      if (st != VP_OK && status[i] == VP_OK) status[i] = st;
      mps_free(out[i]);
      delete out[i];
      out[i] = nullptr;
    }
  return st;
}

int vp_group_stats(const vp_group* g, double* step_ms, double* wait_ms, int64_t* waits, int64_t* launches) {
  if (!g) return VP_EINVAL;
  if (step_ms) *step_ms = g->stat_step_ms;
  if (wait_ms) *wait_ms = g->stat_wait_ms;
  if (waits) *waits = g->stat_waits;
  if (launches) *launches = g->stat_launches;
  return VP_OK;
}

int vp_group_destroy(vp_group* g) {
  if (!g) return VP_EINVAL;
  vp_ctx* ctx = g->ctx;
  if (g->side) cudaStreamSynchronize(g->side);
  cudaStreamSynchronize(ctx->stream);
  for (Member* m : g->mem) free_member(ctx, m);
  g->mem.clear();
  for (Work& w : g->cwork) release_work(ctx, w);
  for (auto* v : {&g->cgrid, &g->csites, &g->crem})
    for (DevBuf& b : *v) release(ctx, b);
  dev_free(ctx, g->d_task, sizeof(TaskDev) * 2 * (size_t)g->cap);
  dev_free(ctx, g->d_we, sizeof(double) * 4 * (size_t)g->cap);
  if (g->h_task) cudaFreeHost(g->h_task);
  if (g->h_init) cudaFreeHost(g->h_init);
  if (g->h_we) cudaFreeHost(g->h_we);
  for (cudaEvent_t e : {g->ev_qf[0], g->ev_qf[1], g->ev_qd[0], g->ev_qd[1], g->ev_fork, g->ev_join})
    if (e) cudaEventDestroy(e);
  if (g->side) cudaStreamDestroy(g->side);
  delete g;
  return VP_OK;
}

}  // extern "C"
