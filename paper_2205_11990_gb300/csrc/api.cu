// C ABI of the MPS Vlasov-Poisson library: contexts, MPS/MPO objects, the
// compression sweeps, the field solve and the RK4 stepper (compression level
// C1).  Host code only orchestrates: every arithmetic step runs in the
// kernels of linalg.cu / mpsops.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <string>
#include <vector>

#include "common.cuh"
#include "mpo_build.hpp"
#include "sim.hpp"

using vp::DevBuf;

namespace vp {

int fail(vp_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

int cuda_fail(vp_ctx* ctx, cudaError_t e, const char* what) {
  return fail(ctx, VP_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void drain_pending(vp_ctx* ctx, bool all) {
  size_t k = 0;
  for (size_t i = 0; i < ctx->pending.size(); ++i) {
    const vp_ctx::PendingFree f = ctx->pending[i];
    bool done = true;
    if (all) {
      cudaEventSynchronize(f.ev);
    } else {
      const cudaError_t q = cudaEventQuery(f.ev);
      if (q == cudaErrorNotReady) {
        (void)cudaGetLastError();  // "not ready" is a status, not an error
        done = false;
      }
    }
    if (done) {
      ctx->freef(f.p, f.bytes, ctx->user);
      ctx->free_events.push_back(f.ev);
    } else {
      ctx->pending[k++] = f;
    }
  }
  ctx->pending.resize(k);
}

void* dev_alloc(vp_ctx* ctx, size_t bytes) {
  if (bytes == 0) bytes = 8;
  if (ctx->alloc) {
    drain_pending(ctx, false);
    return ctx->alloc(bytes, ctx->user);
  }
  void* p = nullptr;
  const cudaError_t e = ctx->pool ? cudaMallocFromPoolAsync(&p, bytes, ctx->pool, ctx->stream)
                                  : cudaMallocAsync(&p, bytes, ctx->stream);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(vp_ctx* ctx, void* p, size_t bytes) {
  if (!p) return;
  if (!ctx->freef) {
    cudaFreeAsync(p, ctx->stream);  // stream-ordered by the runtime's pool
    return;
  }
  cudaEvent_t ev = nullptr;
  if (!ctx->free_events.empty()) {
    ev = ctx->free_events.back();
    ctx->free_events.pop_back();
  } else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
    ev = nullptr;
  }
  if (ev && cudaEventRecord(ev, ctx->stream) == cudaSuccess) {
    ctx->pending.push_back({p, bytes, ev});
  } else {
    cudaStreamSynchronize(ctx->stream);
    ctx->freef(p, bytes, ctx->user);
    if (ev) ctx->free_events.push_back(ev);
  }
}

int reserve(vp_ctx* ctx, DevBuf& b, size_t elems) {
  if (elems <= b.cap && b.p) return VP_OK;
  size_t cap = std::max<size_t>(elems, 64);
  cap = cap + cap / 4;
  void* p = dev_alloc(ctx, cap * sizeof(double));
  if (!p) return fail(ctx, VP_ENOMEM, "device allocation failed");
  dev_free(ctx, b.p, b.cap * sizeof(double));
  b.p = (double*)p;
  b.cap = cap;
  return VP_OK;
}

int reserve_keep(vp_ctx* ctx, DevBuf& b, size_t elems, size_t keep) {
  if (elems <= b.cap && b.p) return VP_OK;
  DevBuf nb;
  VP_TRY(reserve(ctx, nb, elems));
  if (b.p && keep) VP_TRY(launch_copy(ctx, b.p, nb.p, std::min(keep, b.cap)));
  release(ctx, b);
  b = nb;
  return VP_OK;
}

void release(vp_ctx* ctx, DevBuf& b) {
  dev_free(ctx, b.p, b.cap * sizeof(double));
  b.p = nullptr;
  b.cap = 0;
}

int check_launch(vp_ctx* ctx, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, what);
  return VP_OK;
}

static cudaEvent_t next_event(vp_ctx* ctx) {
  if (ctx->ev_used == ctx->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    ctx->ev_pool.push_back(e);
  }
  return ctx->ev_pool[ctx->ev_used++];
}

void prof_begin(vp_ctx* ctx, int cls) {
  if (!ctx->prof_on) return;
  const size_t idx = ctx->ev_used;
  cudaEvent_t e = next_event(ctx);
  if (!e) return;
  cudaEventRecord(e, ctx->stream);
  ctx->prof_marks.push_back({cls, idx, 0, 0, 0});
}

void prof_end(vp_ctx* ctx, int cls, double work, int m, int n, int k) {
  if (!ctx->prof_on) return;
  cudaEvent_t e = next_event(ctx);
  if (!e) return;
  cudaEventRecord(e, ctx->stream);
  if (!ctx->prof_marks.empty()) {
    auto& mk = ctx->prof_marks.back();
    mk.m = m;
    mk.n = n;
    mk.k = k;
  }
  ctx->prof_work[cls] += work;
  ctx->prof_launches[cls] += 1;
}

int AttrOnce::ensure(vp_ctx* ctx, const void* fn, int smem_bytes, bool cluster) {
  static std::mutex mu;
  const int dev = ctx->device;
  const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return VP_OK;
  std::lock_guard<std::mutex> lk(mu);
  if (bit && (done.load(std::memory_order_relaxed) & bit)) return VP_OK;
  if (smem_bytes > 0) VP_CUDA(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes));
  if (cluster) VP_CUDA(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  done.fetch_or(bit, std::memory_order_release);
  return VP_OK;
}

int write_wait_limit(vp_ctx* ctx) {
  VP_CUDA(ctx, cudaMemcpyAsync(&ctx->status->wait_clocks, &ctx->wait_clocks, sizeof(long long),
                               cudaMemcpyHostToDevice, ctx->stream));
  // the source is pageable host memory: the copy has read it on return
  return VP_OK;
}

int sync_status(vp_ctx* ctx) {
  VP_CUDA(ctx, cudaMemcpyAsync(ctx->h_small + 60, &ctx->status->err, sizeof(int), cudaMemcpyDeviceToHost,
                               ctx->stream));
  VP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const int err = ctx->h_small[60];
  if (err == 0) return VP_OK;
  VP_CUDA(ctx, cudaMemsetAsync(ctx->status, 0, sizeof(DevStatus), ctx->stream));
  VP_TRY(write_wait_limit(ctx));
  if (err == 1) return fail(ctx, VP_ETIMEOUT, "a device-side grid barrier gave up waiting");
  if (err == 2) return fail(ctx, VP_ENUMERIC, "NaN or Inf in the input or the singular values");
  return fail(ctx, VP_ENUMERIC, "Jacobi SVD did not converge");
}

// ------------------------------------------------------------ MPS helpers
size_t core_elems(const mps_t* m, int k) { return (size_t)m->r[k] * 2 * m->r[k + 1]; }

int mps_init(vp_ctx* ctx, mps_t* m, int n) {
  m->ctx = ctx;
  m->n = n;
  m->r.assign(n + 1, 1);
  m->core.assign(n, DevBuf{});
  return VP_OK;
}

void mps_free(mps_t* m) {
  for (auto& b : m->core) release(m->ctx, b);
  m->core.clear();
}

static int mps_copy(vp_ctx* ctx, const mps_t* src, mps_t* dst) {
  if (dst->n != src->n) {
    mps_free(dst);
    mps_init(ctx, dst, src->n);
  }
  dst->r = src->r;
  for (int k = 0; k < src->n; ++k) {
    VP_TRY(reserve(ctx, dst->core[k], core_elems(src, k)));
    VP_TRY(launch_copy(ctx, src->core[k].p, dst->core[k].p, core_elems(src, k)));
  }
  return VP_OK;
}

static int read_rank(vp_ctx* ctx, int* r, double* err) {
  VP_CUDA(ctx, cudaMemcpyAsync(ctx->h_small, ctx->d_small, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  VP_CUDA(ctx, cudaMemcpyAsync(ctx->h_smalld, ctx->d_smalld, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  VP_CUDA(ctx, cudaMemcpyAsync(ctx->h_small + 61, &ctx->status->pad2, sizeof(int), cudaMemcpyDeviceToHost,
                               ctx->stream));
  VP_TRY(sync_status(ctx));
  *r = ctx->h_small[0];
  if (err) *err = ctx->h_smalld[0];
  return VP_OK;
}

static thread_local Flops* g_flops = nullptr;
static thread_local double* g_entropy = nullptr;  // per-bond entanglement entropy of the compression running

static double qr_flops(double m, double n) {
  return m >= n ? 2 * m * n * n - 2.0 / 3.0 * n * n * n : 2 * n * m * m - 2.0 / 3.0 * m * m * m;
}

// ------------------------------------------------------------ compression
// QR step at site k: core_k (2 r_k x r_{k+1}) = Q R; core_k <- Q, core_{k+1} <- R core_{k+1}.
static int ensure_side(vp_ctx* ctx) {
  if (ctx->side) return VP_OK;
  VP_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
  VP_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
  VP_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
  for (int b = 0; b < 2; ++b) {
    VP_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_qf[b], cudaEventDisableTiming));
    VP_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_qd[b], cudaEventDisableTiming));
  }
  return VP_OK;
}

// Launches inside the scope go to the side stream with the side scratch.
struct SideScope {
  vp_ctx* c;
  explicit SideScope(vp_ctx* ctx) : c(ctx) { swap_all(); }
  ~SideScope() { swap_all(); }
  void swap_all() {
    std::swap(c->stream, c->side);
    std::swap(c->w_q, c->w_q_side);
    std::swap(c->w_split, c->w_split_side);
    std::swap(c->w_tca, c->w_tca_side);
    std::swap(c->w_tcb, c->w_tcb_side);
    std::swap(c->w_fq, c->w_fq_side);
  }
};

// QR sweep over sites 0..kend-1 (left-canonical form up to site kend): at
// site k the Householder QR of the (2 r_{k-1} x r_k) reshape, R multiplied
// into core k+1 on the context's stream, while Q (the new core k) is formed
// on the side stream; the factor of site k lives in one of two buffers, so
// the Q of site k is formed while site k+1 is factored.  Returns with every Q
// formed (the context's stream waits for the side stream).
static int qr_sweep(vp_ctx* ctx, mps_t* s, int kend) {
  VP_TRY(ensure_side(ctx));
  // On every exit (error paths included) the context's stream waits for the
  // Q formations still in flight: later frees of the factor buffers and
  // writes of the cores are ordered after them.
  struct JoinGuard {
    vp_ctx* c;
    bool busy[2] = {false, false};
    ~JoinGuard() {
      for (int b = 0; b < 2; ++b)
        if (busy[b]) cudaStreamWaitEvent(c->stream, c->ev_qd[b], 0);
    }
  } guard{ctx};
  bool* busy = guard.busy;
  for (int k = 0; k < kend; ++k) {
    const int b = k & 1;
    DevBuf& F = b ? ctx->w_fac_b : ctx->w_fac;
    DevBuf& P = b ? ctx->w_p_b : ctx->w_p;
    if (busy[b]) {  // the Q formation two sites back still reads this buffer
      VP_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_qd[b], 0));
      busy[b] = false;
    }
    const int m = 2 * s->r[k], n = s->r[k + 1], p = std::min(m, n);
    const int nn = 2 * s->r[k + 2];
    VP_TRY(reserve(ctx, F, (size_t)m * n));
    VP_TRY(reserve(ctx, P, (size_t)2 * m + p + 8));
    double* tau = P.p;
    double* vbuf = P.p + p + 8;
    VP_TRY(launch_to_colmajor(ctx, s->core[k].p, m, n, F.p));
    prof_begin(ctx, VP_K_QR);
    VP_TRY(launch_qr_factor(ctx, F.p, m, n, tau, vbuf));
    prof_end(ctx, VP_K_QR, qr_flops(m, n), m, n);
    VP_CUDA(ctx, cudaEventRecord(ctx->ev_qf[b], ctx->stream));
    {
      SideScope side(ctx);
      VP_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_qf[b], 0));
      prof_begin(ctx, VP_K_FORMQ);
      VP_TRY(launch_qr_formq(ctx, F.p, m, n, tau, s->core[k].p));
      prof_end(ctx, VP_K_FORMQ, 4.0 * m * p * p - 4.0 / 3.0 * p * p * p, m, p);
      VP_CUDA(ctx, cudaEventRecord(ctx->ev_qd[b], ctx->stream));
    }
    busy[b] = true;
    VP_TRY(reserve(ctx, ctx->w_gemm, (size_t)p * nn));
    prof_begin(ctx, VP_K_GEMM);
    VP_TRY(launch_gemm_r(ctx, p, nn, n, F.p, m, s->core[k + 1].p, nn, ctx->w_gemm.p, nn));
    prof_end(ctx, VP_K_GEMM, 2.0 * p * n * nn, p, nn, n);
    std::swap(s->core[k + 1], ctx->w_gemm);
    s->r[k + 1] = p;
    if (g_flops) {
      g_flops->qr += qr_flops(m, n);
      g_flops->formq += 4.0 * m * p * p - 4.0 / 3.0 * p * p * p;
      g_flops->gemm += 2.0 * p * n * nn;
    }
  }
  for (int b = 0; b < 2; ++b)
    if (busy[b]) {
      busy[b] = false;
      VP_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_qd[b], 0));
    }
  return VP_OK;
}

// SVD step at site k >= 1 of a left-canonical MPS whose right part is
// already right-canonical: M = core_k (r_k x 2 r_{k+1}); keep r singular
// triplets (truncation rule of the truncation-error equation).
//
// The SVD is one-sided Jacobi on a preconditioned square factor.  With A = M
// (tall) or M^T (wide), q = min(r_k, 2 r_{k+1}):  A Pi = Q1 R1 (columns
// ordered by decreasing norm, Householder QR), R1^T = Q2 L^T (second QR),
// then Jacobi on the rows of the lower-triangular L (graded, so it converges
// in far fewer sweeps than on M itself).  L = U_L S V_L^T gives
//   tall: M = Q1 U_L S (Pi Q2 V_L)^T  ->  core_{k-1} <- P Q1 U_L S,
//         core_k <- (V_L^T Q2^T) with columns scattered back by Pi;
//   wide: M = Pi Q2 V_L S (Q1 U_L)^T ->  core_k <- U_L^T Q1^T,
//         core_{k-1} <- P Pi (Q2 V_L S).
static int svd_site(vp_ctx* ctx, mps_t* s, int k, int chi, double tol, double* err_out, double* sig_out = nullptr) {
  const int m = s->r[k];
  const int c = 2 * s->r[k + 1];
  const int pl = 2 * s->r[k - 1];  // rows of the previous core viewed as (2 r_{k-1} x r_k)
  const bool tall = m >= c;
  const int q = tall ? c : m;  // square factor size
  const int p = tall ? m : c;  // long side of A
  VP_TRY(reserve(ctx, ctx->w_piv, (size_t)q / 2 + 8));
  int* piv = (int*)ctx->w_piv.p;
  VP_TRY(launch_norm_order(ctx, s->core[k].p, m, c, tall ? 1 : 0, piv));
  // first QR: A Pi = Q1 R1
  VP_TRY(reserve(ctx, ctx->w_fac, (size_t)p * q));
  VP_TRY(reserve(ctx, ctx->w_p, (size_t)2 * p + q + 8));
  VP_TRY(launch_gather_cm(ctx, s->core[k].p, m, c, piv, tall ? 1 : 0, ctx->w_fac.p));
  prof_begin(ctx, VP_K_QR);
  VP_TRY(launch_qr_factor(ctx, ctx->w_fac.p, p, q, ctx->w_p.p, ctx->w_p.p + q + 8));
  prof_end(ctx, VP_K_QR, qr_flops(p, q), p, q);
  VP_TRY(reserve(ctx, ctx->w_q1, (size_t)p * q));
  // second QR: R1^T = Q2 L^T (R1 row-major is R1^T column-major)
  VP_TRY(reserve(ctx, ctx->w_r, (size_t)q * q));
  VP_TRY(launch_qr_getr(ctx, ctx->w_fac.p, p, q, ctx->w_r.p));
  VP_TRY(reserve(ctx, ctx->w_p2, (size_t)3 * q + 8));
  prof_begin(ctx, VP_K_QR);
  VP_TRY(launch_qr_factor(ctx, ctx->w_r.p, q, q, ctx->w_p2.p, ctx->w_p2.p + q + 8));
  prof_end(ctx, VP_K_QR, qr_flops(q, q), q, q);
  VP_TRY(reserve(ctx, ctx->w_q2, (size_t)q * q));
  // Q1, Q2 (and, tall, P Q1) only feed the outputs: form them on the side
  // stream while the Jacobi SVD runs.  Their scratch is reserved up front so
  // nothing is reallocated while the two streams run.
  if (tall) VP_TRY(reserve(ctx, ctx->w_tmp2, (size_t)pl * q));
  VP_TRY(ensure_side(ctx));
  VP_TRY(reserve(ctx, ctx->w_q_side, (size_t)std::max(p, q) * q));
  VP_TRY(reserve(ctx, ctx->w_split_side, (size_t)pl * q * 33));
  VP_CUDA(ctx, cudaEventRecord(ctx->ev_fork, ctx->stream));
  VP_CUDA(ctx, cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
  {
    SideScope side(ctx);
    prof_begin(ctx, VP_K_FORMQ);
    VP_TRY(launch_qr_formq(ctx, ctx->w_fac.p, p, q, ctx->w_p.p, ctx->w_q1.p));
    prof_end(ctx, VP_K_FORMQ, 4.0 * p * q * q - 4.0 / 3.0 * q * q * q, p, q);
    prof_begin(ctx, VP_K_FORMQ);
    VP_TRY(launch_qr_formq(ctx, ctx->w_r.p, q, q, ctx->w_p2.p, ctx->w_q2.p));
    prof_end(ctx, VP_K_FORMQ, 8.0 / 3.0 * q * q * q, q, q);
    if (tall) VP_TRY(launch_gemm(ctx, pl, q, m, 1.0, s->core[k - 1].p, m, ctx->w_q1.p, q, ctx->w_tmp2.p, q));
  }
  VP_CUDA(ctx, cudaEventRecord(ctx->ev_join, ctx->side));
  // every exit from here on makes the context's stream wait for the side
  // stream's products (the normal path joins before the outputs, again below)
  struct SideJoin {
    vp_ctx* c;
    ~SideJoin() { cudaStreamWaitEvent(c->stream, c->ev_join, 0); }
  } side_join{ctx};
  VP_TRY(reserve(ctx, ctx->w_tmp, (size_t)q * q));
  double* X = ctx->w_tmp.p;
  VP_TRY(launch_lower_from_upper(ctx, ctx->w_r.p, q, X));
  // Jacobi on the rows of L.  Tall case: no rotation accumulator; U_L S = L V_L
  // is recovered afterwards from a saved copy of L.
  double* Lsave = nullptr;
  if (tall) {
    VP_TRY(reserve(ctx, ctx->w_l, (size_t)q * q));
    VP_TRY(launch_copy(ctx, X, ctx->w_l.p, (size_t)q * q));
    Lsave = ctx->w_l.p;
  } else {
    VP_TRY(reserve(ctx, ctx->w_j, (size_t)q * q));
  }
  VP_CUDA(ctx, cudaMemsetAsync(ctx->status->rot, 0, sizeof(ctx->status->rot), ctx->stream));
  prof_begin(ctx, VP_K_JACOBI);
  VP_TRY(launch_jacobi_rows(ctx, X, q, q, tall ? nullptr : ctx->w_j.p, tol >= 1e-13));
  prof_end(ctx, VP_K_JACOBI, 0.0, q, q);
  const size_t jac_mark = ctx->prof_on && !ctx->prof_marks.empty() ? ctx->prof_marks.size() - 1 : (size_t)-1;
  VP_TRY(reserve(ctx, ctx->w_vec, (size_t)2 * q + 8));
  int* perm = (int*)ctx->w_vec.p;
  double* sigma = ctx->w_vec.p + (q + 1) / 2 + 4;
  prof_begin(ctx, VP_K_SELECT);
  VP_TRY(launch_select(ctx, X, q, q, chi, tol, perm, sigma, ctx->d_small, ctx->d_smalld));
  prof_end(ctx, VP_K_SELECT, 0.0, q, q);
  int r = 1;
  double err = 0.0;
  VP_TRY(read_rank(ctx, &r, &err));
  if (err_out) *err_out = err;
  if (g_entropy) g_entropy[k - 1] = ctx->h_smalld[1];
  if (sig_out) VP_TRY(launch_copy(ctx, sigma, sig_out, (size_t)r));
  const double jac = q > 1 ? (double)ctx->h_small[61] * 0.5 * q * (q - 1) * (6.0 * q + (tall ? 0.0 : 4.0 * q)) : 0.0;
  if (ctx->prof_on) ctx->prof_work[VP_K_JACOBI] += jac;
  if (jac_mark != (size_t)-1 && jac_mark < ctx->prof_marks.size()) ctx->prof_marks[jac_mark].k = ctx->h_small[61];
  double gem = 0.0;
  VP_TRY(reserve(ctx, ctx->w_a, (size_t)r * q + 8));
  VP_TRY(reserve(ctx, ctx->w_b, (size_t)q * r + 8));
  VP_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));
  prof_begin(ctx, VP_K_GEMM);
  if (tall) {
    // P1 = P Q1 (pl x q); core_{k-1} <- P1 (U_L S); core_k <- scatter(V_L^T Q2^T)
    VP_TRY(launch_svd_outputs(ctx, X, nullptr, q, q, r, perm, sigma, ctx->w_a.p, nullptr));
    VP_TRY(launch_gemm_bt(ctx, q, r, q, Lsave, q, ctx->w_a.p, q, ctx->w_b.p, r));  // U_L S = L V_L
    VP_TRY(reserve(ctx, ctx->w_gemm, (size_t)pl * r));
    VP_TRY(launch_gemm(ctx, pl, r, q, 1.0, ctx->w_tmp2.p, q, ctx->w_b.p, r, ctx->w_gemm.p, r));
    VP_TRY(reserve(ctx, ctx->w_c, (size_t)r * q));
    VP_TRY(launch_gemm_bt(ctx, r, q, q, ctx->w_a.p, q, ctx->w_q2.p, q, ctx->w_c.p, q));
    VP_TRY(reserve(ctx, s->core[k], (size_t)r * c));
    VP_TRY(launch_scatter(ctx, ctx->w_c.p, r, q, piv, 1, s->core[k].p));
    gem = 2.0 * pl * q * m + 2.0 * pl * r * q + 2.0 * r * q * q + 2.0 * q * q * r;
  } else {
    // core_k <- U_L^T Q1^T (r x c); core_{k-1} <- P Pi (Q2 V_L S)
    VP_TRY(launch_svd_outputs_wide(ctx, X, ctx->w_j.p, q, r, perm, ctx->w_a.p, ctx->w_b.p));
    VP_TRY(reserve(ctx, s->core[k], (size_t)r * c));
    VP_TRY(launch_gemm_bt(ctx, r, c, m, ctx->w_a.p, m, ctx->w_q1.p, m, s->core[k].p, c));
    VP_TRY(reserve(ctx, ctx->w_c, (size_t)m * r));
    VP_TRY(launch_gemm(ctx, m, r, m, 1.0, ctx->w_q2.p, m, ctx->w_b.p, r, ctx->w_c.p, r));
    VP_TRY(reserve(ctx, ctx->w_tmp2, (size_t)m * r));
    VP_TRY(launch_scatter(ctx, ctx->w_c.p, m, r, piv, 0, ctx->w_tmp2.p));
    VP_TRY(reserve(ctx, ctx->w_gemm, (size_t)pl * r));
    VP_TRY(launch_gemm(ctx, pl, r, m, 1.0, s->core[k - 1].p, m, ctx->w_tmp2.p, r, ctx->w_gemm.p, r));
    gem = 2.0 * r * c * m + 2.0 * m * r * m + 2.0 * pl * r * m;
  }
  prof_end(ctx, VP_K_GEMM, gem, q, r, pl);
  std::swap(s->core[k - 1], ctx->w_gemm);
  s->r[k] = r;
  if (g_flops) {
    g_flops->qr += qr_flops(p, q) + qr_flops(q, q);
    g_flops->formq += 4.0 * p * q * q - 4.0 / 3.0 * q * q * q + 8.0 / 3.0 * q * q * q;
    g_flops->jacobi += jac;
    g_flops->gemm += gem;
  }
  return VP_OK;
}

// Tolerance of the bonds inside the (x_j, v_j) pairs of the IG ordering:
// three orders below the step's 1e-10, so the pair cores are represented
// exactly to FP64 working accuracy.
constexpr double kPairTol = 1e-13;

static int svd_sweep(vp_ctx* ctx, mps_t* s, int chi, double tol, double* errs) {
  for (int k = s->n - 1; k >= 1; --k) {
    // site k splits the bond after site k-1; in the IG ordering the bonds
    // after the even sites (2j: x_j | v_j) lie inside a pair
    const bool inner = ctx->grouped && (k & 1);
    VP_TRY(svd_site(ctx, s, k, inner ? 1 << 30 : chi, inner ? std::min(tol, kPairTol) : tol,
                    errs ? errs + (k - 1) : nullptr));
  }
  return VP_OK;
}

// Right-canonical site k (k >= 1): M = core_k as (r_{k-1} x 2 r_k) = L Q with
// orthonormal rows Q, from the Householder QR of M^T (whose column-major
// layout is M's row-major one); core_k <- Q, core_{k-1} <- core_{k-1} L.
static int lq_site(vp_ctx* ctx, mps_t* s, int k) {
  const int m = 2 * s->r[k + 1], n = s->r[k], p = std::min(m, n);
  const int rows = 2 * s->r[k - 1];
  VP_TRY(reserve(ctx, ctx->w_fac, (size_t)m * n));
  VP_TRY(reserve(ctx, ctx->w_p, (size_t)2 * m + p + 8));
  VP_TRY(launch_copy(ctx, s->core[k].p, ctx->w_fac.p, (size_t)m * n));
  double* tau = ctx->w_p.p;
  prof_begin(ctx, VP_K_QR);
  VP_TRY(launch_qr_factor(ctx, ctx->w_fac.p, m, n, tau, ctx->w_p.p + p + 8));
  prof_end(ctx, VP_K_QR, qr_flops(m, n), m, n);
  VP_TRY(reserve(ctx, ctx->w_q1, (size_t)m * p));
  prof_begin(ctx, VP_K_FORMQ);
  VP_TRY(launch_qr_formq(ctx, ctx->w_fac.p, m, n, tau, ctx->w_q1.p));
  prof_end(ctx, VP_K_FORMQ, 4.0 * m * p * p - 4.0 / 3.0 * p * p * p, m, p);
  VP_TRY(reserve(ctx, ctx->w_r, (size_t)p * n));
  VP_TRY(launch_qr_getr(ctx, ctx->w_fac.p, m, n, ctx->w_r.p));
  VP_TRY(reserve(ctx, ctx->w_tmp, (size_t)p * m));
  VP_TRY(launch_to_colmajor(ctx, ctx->w_q1.p, m, p, ctx->w_tmp.p));  // Q^T, row-major (p x m)
  VP_TRY(reserve(ctx, ctx->w_gemm, (size_t)rows * p));
  prof_begin(ctx, VP_K_GEMM);
  VP_TRY(launch_gemm_bt(ctx, rows, p, n, s->core[k - 1].p, n, ctx->w_r.p, n, ctx->w_gemm.p, p));
  prof_end(ctx, VP_K_GEMM, 2.0 * rows * p * n, rows, p, n);
  std::swap(s->core[k], ctx->w_tmp);
  std::swap(s->core[k - 1], ctx->w_gemm);
  s->r[k] = p;
  return VP_OK;
}

// Modified centre-bond-first compression (SI "Modified Compression Scheme")
// about the bond between sites split-1 and split (the x / v cut of a
// sequential ordering):
//  1. sites right of split right-canonical (LQ), sites left of it
//     left-canonical (QR, R into core split);
//  2. the SVD of core split truncates the centre bond: core split-1 takes
//     U S, core split V^T -- the same U and S as the SVD of the centre bond
//     matrix, since core split = C Q with Q orthonormal rows;
//  3. S^{-1} S inserted: core split scaled by S (the kept values), S^{-1}
//     held back, so each half sees an orthonormal other half;
//  4. the x half swept from the centre to the left end (right-to-left SVD
//     steps), 5. the v half from the centre to the right end: the same
//     steps on the v half read back to front (cores transposed), 6. S^{-1}
//     absorbed into core split.
static int compress_modified(vp_ctx* ctx, mps_t* s, int split, int chi, double tol, double* errs) {
  const int n = s->n;
  if (split < 1 || split >= n) return fail(ctx, VP_EINVAL, "modified compression: bad split");
  for (int k = n - 1; k > split; --k) VP_TRY(lq_site(ctx, s, k));
  VP_TRY(qr_sweep(ctx, s, split));
  VP_TRY(reserve(ctx, ctx->w_sig, (size_t)s->r[split] + 8));
  VP_TRY(svd_site(ctx, s, split, chi, tol, errs ? errs + split - 1 : nullptr, ctx->w_sig.p));
  const int rc = s->r[split];
  for (int k = split - 1; k >= 1; --k) VP_TRY(svd_site(ctx, s, k, chi, tol, errs ? errs + k - 1 : nullptr));
  VP_TRY(launch_scale_rows(ctx, s->core[split].p, rc, 2 * s->r[split + 1], ctx->w_sig.p, 0));
  // v half: the chain split .. n-1 read back to front
  const int mv = n - split;
  if (mv > 1) {
    mps_t rv;
    rv.ctx = ctx;
    rv.n = mv;
    rv.r.assign(mv + 1, 1);
    rv.core.assign(mv, DevBuf{});
    for (int j = 0; j < mv; ++j) {
      const int k = n - 1 - j;
      rv.r[j + 1] = s->r[k];
      VP_TRY(reserve(ctx, rv.core[j], (size_t)s->r[k] * 2 * s->r[k + 1]));
      VP_TRY(launch_core_transpose(ctx, s->core[k].p, s->r[k], s->r[k + 1], rv.core[j].p));
    }
    rv.r[0] = s->r[n];
    std::vector<double> e(mv, 0.0), ee(mv, 0.0);
    double* ent = g_entropy;
    g_entropy = ent ? ee.data() : nullptr;
    for (int j = mv - 1; j >= 1; --j) {
      const int st = svd_site(ctx, &rv, j, chi, tol, &e[j - 1]);
      if (st != VP_OK) {
        g_entropy = ent;
        for (auto& b : rv.core) release(ctx, b);
        return st;
      }
    }
    g_entropy = ent;
    for (int j = 1; j < mv; ++j) {  // rv bond j-1 is the bond after site n-1-j
      if (errs) errs[n - 1 - j] = e[j - 1];
      if (ent) ent[n - 1 - j] = ee[j - 1];
    }
    for (int j = 0; j < mv; ++j) {
      const int k = n - 1 - j;
      s->r[k] = rv.r[j + 1];
      VP_TRY(reserve(ctx, s->core[k], (size_t)rv.r[j + 1] * 2 * rv.r[j]));
      VP_TRY(launch_core_transpose(ctx, rv.core[j].p, rv.r[j], rv.r[j + 1], s->core[k].p));
    }
    for (auto& b : rv.core) release(ctx, b);
  }
  return launch_scale_rows(ctx, s->core[split].p, rc, 2 * s->r[split + 1], ctx->w_sig.p, 1);
}

int compress(vp_ctx* ctx, mps_t* s, int chi, double tol, double* errs) {
  if (ctx->modified_split > 0 && ctx->modified_split < s->n)
    return compress_modified(ctx, s, ctx->modified_split, chi, tol, errs);
  VP_TRY(qr_sweep(ctx, s, s->n - 1));
  return svd_sweep(ctx, s, chi, tol, errs);
}

// Exact left-canonical MPS of a site-ordered device vector (2^n entries, in
// ctx->w_tmp) by a chain of QR factorisations of reshapes, then the SVD sweep.
static int from_vector(vp_ctx* ctx, mps_t* s, int n, const double* vec, int chi, double tol) {
  mps_init(ctx, s, n);
  DevBuf rem;
  const size_t N = (size_t)1 << n;
  VP_TRY(reserve(ctx, rem, N));
  VP_TRY(launch_copy(ctx, vec, rem.p, N));
  int r = 1;
  for (int k = 0; k + 1 < n; ++k) {
    const int m = 2 * r;
    const size_t cols = N >> (k + 1);
    if (cols > (size_t)1 << 30) return fail(ctx, VP_ECAPACITY, "vector too long");
    const int nc = (int)cols, p = (int)std::min<size_t>(m, cols);
    VP_TRY(reserve(ctx, ctx->w_fac, (size_t)m * nc));
    VP_TRY(reserve(ctx, ctx->w_p, (size_t)2 * m + p + 8));
    VP_TRY(launch_to_colmajor(ctx, rem.p, m, nc, ctx->w_fac.p));
    VP_TRY(launch_qr_factor(ctx, ctx->w_fac.p, m, nc, ctx->w_p.p, ctx->w_p.p + p + 8));
    VP_TRY(reserve(ctx, s->core[k], (size_t)m * p));
    VP_TRY(launch_qr_formq(ctx, ctx->w_fac.p, m, nc, ctx->w_p.p, s->core[k].p));
    VP_TRY(launch_qr_getr(ctx, ctx->w_fac.p, m, nc, rem.p));
    s->r[k + 1] = p;
    r = p;
  }
  VP_TRY(reserve(ctx, s->core[n - 1], (size_t)2 * r));
  VP_TRY(launch_copy(ctx, rem.p, s->core[n - 1].p, (size_t)2 * r));
  release(ctx, rem);
  if (n > 1) VP_TRY(svd_sweep(ctx, s, chi, tol, nullptr));
  return VP_OK;
}

// Dense vector (2^n, site bits) of an MPS into dev (capacity 2^n).
static int to_dense_dev(vp_ctx* ctx, const mps_t* s, DevBuf& out) {
  const int n = s->n;
  DevBuf a, b;
  VP_TRY(reserve(ctx, a, core_elems(s, 0)));
  VP_TRY(launch_copy(ctx, s->core[0].p, a.p, core_elems(s, 0)));
  size_t rows = 2;
  for (int k = 1; k < n; ++k) {
    const int rk = s->r[k], rn = s->r[k + 1];
    VP_TRY(reserve(ctx, b, rows * 2 * rn));
    if (rows > (size_t)1 << 26) return fail(ctx, VP_ECAPACITY, "to_dense: too many sites");
    VP_TRY(launch_gemm(ctx, (int)rows, 2 * rn, rk, 1.0, a.p, rk, s->core[k].p, 2 * rn, b.p, 2 * rn));
    std::swap(a, b);
    rows *= 2;
  }
  std::swap(out, a);
  release(ctx, a);
  release(ctx, b);
  return VP_OK;
}

// ------------------------------------------------------------ density
bool xdesc(const vp_layout* L) { return L->mapping == VP_SEQ_S2; }
bool vdesc(const vp_layout* L) { return L->mapping == VP_SEQ_S3; }
bool interleaved(const vp_layout* L) {
  return L->mapping == VP_INTERLEAVED || L->mapping == VP_INTERLEAVED_GROUPED;
}
bool grouped(const vp_layout* L) { return L->mapping == VP_INTERLEAVED_GROUPED; }

std::vector<int> site_dims(const vp_layout* L) {
  std::vector<int> d;
  if (!interleaved(L)) {
    for (int b = 0; b < L->nx; ++b) d.push_back(0);
    for (int b = 0; b < L->nv; ++b) d.push_back(1);
  } else {
    for (int b = 0; b < std::max(L->nx, L->nv); ++b) {
      if (b < L->nx) d.push_back(0);
      if (b < L->nv) d.push_back(1);
    }
  }
  return d;
}

// rho (2^nx, device) = dv * contraction of every v site with [1, 1], then
// expansion of the remaining x MPS (SI "Integration").
static int density(vp_ctx* ctx, const vp_layout* L, const mps_t* f, double* rho) {
  const std::vector<int> dims = site_dims(L);
  const double dv = (L->vmax - L->vmin) / (double)((1 << L->nv) - 1);
  // pending (pl x pr) matrix of contracted v sites not yet absorbed
  DevBuf pend, tmp, T;
  bool have_pend = false;
  int pend_l = 1, pend_r = 1;
  std::vector<DevBuf> xc;  // x cores after absorption
  std::vector<int> xr;     // x bonds
  xr.push_back(1);
  for (int k = 0; k < f->n; ++k) {
    const int rl = f->r[k], rr = f->r[k + 1];
    if (dims[k] == 1) {
      VP_TRY(reserve(ctx, T, (size_t)rl * rr));
      VP_TRY(launch_phys_sum(ctx, f->core[k].p, rl, rr, T.p));
      if (!have_pend) {
        std::swap(pend, T);
        pend_l = rl;
        pend_r = rr;
        have_pend = true;
      } else {
        VP_TRY(reserve(ctx, tmp, (size_t)pend_l * rr));
        VP_TRY(launch_gemm(ctx, pend_l, rr, rl, 1.0, pend.p, rl, T.p, rr, tmp.p, rr));
        std::swap(pend, tmp);
        pend_r = rr;
      }
    } else {
      DevBuf c;
      if (have_pend) {
        VP_TRY(reserve(ctx, c, (size_t)pend_l * 2 * rr));
        VP_TRY(launch_gemm(ctx, pend_l, 2 * rr, rl, 1.0, pend.p, rl, f->core[k].p, 2 * rr, c.p, 2 * rr));
        have_pend = false;
        xr.back() = pend_l;  // left bond of this x core is the pending left bond
      } else {
        VP_TRY(reserve(ctx, c, (size_t)rl * 2 * rr));
        VP_TRY(launch_copy(ctx, f->core[k].p, c.p, (size_t)rl * 2 * rr));
      }
      xc.push_back(c);
      xr.push_back(rr);
    }
  }
  if (have_pend) {  // trailing v sites: absorb into the last x core on its right
    DevBuf& last = xc.back();
    const int lx = xr[xr.size() - 2], rx = xr.back();
    VP_TRY(reserve(ctx, tmp, (size_t)lx * 2 * pend_r));
    VP_TRY(launch_gemm(ctx, lx * 2, pend_r, rx, 1.0, last.p, rx, pend.p, pend_r, tmp.p, pend_r));
    std::swap(last, tmp);
    xr.back() = pend_r;
  }
  // expand
  mps_t xm;
  mps_init(ctx, &xm, (int)xc.size());
  xm.r = xr;
  for (size_t i = 0; i < xc.size(); ++i) xm.core[i] = xc[i];
  DevBuf dense;
  VP_TRY(to_dense_dev(ctx, &xm, dense));
  const size_t Nx = (size_t)1 << L->nx;
  if (xdesc(L))  // the expansion is indexed by the x bits in site order: undo the bit reversal
    VP_TRY(launch_permute_to_sites(ctx, dense.p, L->nx, 0, VP_SEQ_S2, rho, 1));
  else
    VP_TRY(launch_copy(ctx, dense.p, rho, Nx));
  VP_TRY(launch_scale(ctx, rho, Nx, dv));
  release(ctx, dense);
  mps_free(&xm);
  release(ctx, pend);
  release(ctx, tmp);
  release(ctx, T);
  return VP_OK;
}

bool layout_ok(const vp_layout* L) {
  return L && L->nx >= 2 && L->nv >= 2 && L->nx <= 14 && L->nv <= 14 &&
         L->mapping >= VP_SEQ && L->mapping <= VP_INTERLEAVED_GROUPED &&
         (L->mapping != VP_INTERLEAVED_GROUPED || L->nx == L->nv) && L->xmax > L->xmin && L->vmax > L->vmin &&
         std::fabs(L->vmin + L->vmax) <= 1e-12 * std::fabs(L->vmax);
}

}  // namespace vp

extern "C" int vp_ctx_create(void* cuda_stream, vp_alloc_fn alloc, vp_free_fn free_fn, void* user, vp_ctx** out);

namespace vp {
// A context on its own non-blocking stream with the library's stream-ordered
// allocator, for work that runs concurrently with the parent's stream.
static vp_ctx* ctx_child(vp_ctx* parent) {
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
  vp_ctx* c = nullptr;
  if (vp_ctx_create(st, nullptr, nullptr, nullptr, &c) != VP_OK) {
    cudaStreamDestroy(st);
    return nullptr;
  }
  c->owns_stream = true;
  c->wait_clocks = parent->wait_clocks;
  if (write_wait_limit(c) != VP_OK) {
    vp_ctx_destroy(c);
    return nullptr;
  }
  parent->children.push_back(c);
  return c;
}
}  // namespace vp

// ====================================================================== ABI
using namespace vp;

extern "C" {

int vp_ctx_create(void* cuda_stream, vp_alloc_fn alloc, vp_free_fn free_fn, void* user, vp_ctx** out) {
  if (!out || ((alloc == nullptr) != (free_fn == nullptr))) return VP_EINVAL;
  *out = nullptr;
  int dev = 0, count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) return VP_ECUDA;
  if (cudaGetDevice(&dev) != cudaSuccess) return VP_ECUDA;
  vp_ctx* c = new (std::nothrow) vp_ctx();
  if (!c) return VP_ENOMEM;
  c->device = dev;
  c->stream = (cudaStream_t)cuda_stream;
  c->alloc = alloc;
  c->freef = free_fn;
  c->user = user;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    delete c;
    return VP_ECUDA;
  }
  c->num_sms = prop.multiProcessorCount;
  if (!alloc) {
    // a pool of this context's own that keeps freed memory for reuse (the
    // device's default pool returns it to the system at every synchronise,
    // and the sweeps synchronise once per SVD site)
    cudaMemPoolProps pp = {};
    pp.allocType = cudaMemAllocationTypePinned;
    pp.handleTypes = cudaMemHandleTypeNone;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = dev;
    if (cudaMemPoolCreate(&c->pool, &pp) != cudaSuccess) {
      delete c;
      return VP_ECUDA;
    }
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  c->cluster_size = vp::probe_cluster_size();
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop) {
    delete c;
    return VP_ECUDA;
  }
  c->status = (DevStatus*)dev_alloc(c, sizeof(DevStatus));
  c->d_small = (int*)dev_alloc(c, 64 * sizeof(int));
  c->d_smalld = (double*)dev_alloc(c, 64 * sizeof(double));
  if (!c->status || !c->d_small || !c->d_smalld || cudaMallocHost(&c->h_small, 64 * sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&c->h_smalld, 64 * sizeof(double)) != cudaSuccess) {
    delete c;
    return VP_ENOMEM;
  }
  cudaMemsetAsync(c->status, 0, sizeof(DevStatus), c->stream);
  if (write_wait_limit(c) != VP_OK || cudaStreamSynchronize(c->stream) != cudaSuccess) {
    delete c;
    return VP_ECUDA;
  }
  *out = c;
  return VP_OK;
}

int vp_ctx_destroy(vp_ctx* c) {
  if (!c) return VP_EINVAL;
  cudaStreamSynchronize(c->stream);
  for (DevBuf* b : {&c->w_fac, &c->w_q, &c->w_gemm, &c->w_j, &c->w_p, &c->w_tmp, &c->w_tmp2, &c->w_vec, &c->w_split,
                    &c->w_piv, &c->w_q1, &c->w_q2, &c->w_r, &c->w_p2, &c->w_a, &c->w_b, &c->w_c, &c->w_l,
                    &c->w_q_side, &c->w_split_side, &c->w_tca, &c->w_tcb, &c->w_tca_side, &c->w_tcb_side,
                    &c->w_qrv, &c->w_qrc, &c->w_fq, &c->w_fq_side, &c->w_fac_b, &c->w_p_b,
                    &c->w_sig, &c->w_wq, &c->w_wr})
    release(c, *b);
  for (auto& b : c->w_chain) release(c, b);
  dev_free(c, c->status, sizeof(DevStatus));
  dev_free(c, c->d_small, 64 * sizeof(int));
  dev_free(c, c->d_smalld, 64 * sizeof(double));
  cudaStreamSynchronize(c->stream);
  if (c->side) cudaStreamSynchronize(c->side);
  if (c->freef) drain_pending(c, true);
  for (cudaEvent_t e : c->free_events) cudaEventDestroy(e);
  cudaFreeHost(c->h_small);
  cudaFreeHost(c->h_smalld);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  for (cudaEvent_t e : {c->ev_qf[0], c->ev_qf[1], c->ev_qd[0], c->ev_qd[1]})
    if (e) cudaEventDestroy(e);
  if (c->owns_stream) cudaStreamDestroy(c->stream);
  // memory still outstanding (frees not yet completed) returns when they are
  if (c->pool) cudaMemPoolDestroy(c->pool);
  delete c;
  return VP_OK;
}

const char* vp_last_error(const vp_ctx* c) { return c ? c->err.c_str() : "null context"; }

int vp_ctx_set_wait_limit(vp_ctx* c, long long clocks) {
  if (!c || clocks < 0) return VP_EINVAL;
  c->wait_clocks = clocks > 0 ? clocks : kDefaultWaitClocks;
  VP_TRY(write_wait_limit(c));
  for (vp_ctx* ch : c->children) VP_TRY(vp_ctx_set_wait_limit(ch, clocks));
  VP_CUDA(c, cudaStreamSynchronize(c->stream));
  return VP_OK;
}

int vp_profile_enable(vp_ctx* c, int on) {
  if (!c) return VP_EINVAL;
  for (vp_ctx* ch : c->children) vp_profile_enable(ch, on);
  cudaStreamSynchronize(c->stream);
  c->prof_on = on != 0;
  c->ev_used = 0;
  c->prof_marks.clear();
  for (int k = 0; k < VP_K_COUNT; ++k) {
    c->prof_work[k] = 0.0;
    c->prof_launches[k] = 0;
  }
  return VP_OK;
}

int vp_profile_read(vp_ctx* c, int cls, double* ms, int64_t* launches, double* work) {
  if (!c || cls < 0 || cls >= VP_K_COUNT) return VP_EINVAL;
  VP_CUDA(c, cudaStreamSynchronize(c->stream));
  double t = 0.0;
  for (auto& m : c->prof_marks) {
    if (m.cls != cls) continue;
    float x = 0.f;
    VP_CUDA(c, cudaEventElapsedTime(&x, c->ev_pool[m.ev], c->ev_pool[m.ev + 1]));
    t += x;
  }
  double wk = c->prof_work[cls];
  int64_t nl = c->prof_launches[cls];
  for (vp_ctx* ch : c->children) {
    double t2 = 0.0, w2 = 0.0;
    int64_t n2 = 0;
    VP_TRY(vp_profile_read(ch, cls, &t2, &n2, &w2));
    t += t2;
    wk += w2;
    nl += n2;
  }
  if (ms) *ms = t;
  if (launches) *launches = nl;
  if (work) *work = wk;
  return VP_OK;
}

int vp_profile_trace(vp_ctx* c, vp_trace_rec* out, int cap, int* n_out) {
  if (!c || (!out && cap > 0) || cap < 0 || !n_out) return VP_EINVAL;
  VP_CUDA(c, cudaStreamSynchronize(c->stream));
  if (c->side) VP_CUDA(c, cudaStreamSynchronize(c->side));
  int n = 0;
  for (auto& m : c->prof_marks) {
    if (n < cap) {
      float x = 0.f;
      VP_CUDA(c, cudaEventElapsedTime(&x, c->ev_pool[m.ev], c->ev_pool[m.ev + 1]));
      out[n] = vp_trace_rec{m.cls, m.m, m.n, m.k, (double)x};
    }
    ++n;
  }
  for (vp_ctx* ch : c->children) {
    int n2 = 0;
    VP_TRY(vp_profile_trace(ch, out ? out + std::min(n, cap) : nullptr, std::max(0, cap - n), &n2));
    n += n2;
  }
  *n_out = n;
  return VP_OK;
}

int64_t vp_kernel_launches(const vp_ctx* c) {
  if (!c) return 0;
  int64_t n = c->launches;
  for (const vp_ctx* ch : c->children) n += vp_kernel_launches(ch);
  return n;
}

// ------------------------------------------------------------------- MPS
int mps_create(vp_ctx* ctx, const vp_layout* L, const double* f, int f_on_device, int chi, double tol,
               mps_t** out) {
  if (!ctx || !out || !f || chi < 1 || tol < 0) return fail(ctx, VP_EINVAL, "mps_create: bad argument");
  if (!layout_ok(L)) return fail(ctx, VP_EINVAL, "mps_create: unsupported layout");
  const int n = L->nx + L->nv;
  const size_t N = (size_t)1 << n;
  DevBuf grid, sites;
  VP_TRY(reserve(ctx, grid, N));
  VP_TRY(reserve(ctx, sites, N));
  VP_CUDA(ctx, cudaMemcpyAsync(grid.p, f, N * sizeof(double),
                               f_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
  VP_TRY(launch_check_finite(ctx, grid.p, N));
  VP_TRY(launch_permute_to_sites(ctx, grid.p, L->nx, L->nv, L->mapping, sites.p, 0));
  mps_t* m = new mps_t();
  const int g0 = ctx->grouped;
  ctx->grouped = grouped(L) ? 1 : 0;
  int s = from_vector(ctx, m, n, sites.p, chi, tol);
  ctx->grouped = g0;
  release(ctx, grid);
  release(ctx, sites);
  if (s == VP_OK) s = sync_status(ctx);
  if (s != VP_OK) {
    mps_free(m);
    delete m;
    return s;
  }
  *out = m;
  return VP_OK;
}

int mps_create_cores(vp_ctx* ctx, int n, const int* ranks, const double* cores, mps_t** out) {
  if (!ctx || n < 1 || !ranks || !cores || !out || ranks[0] != 1 || ranks[n] != 1)
    return fail(ctx, VP_EINVAL, "mps_create_cores: bad argument");
  mps_t* m = new mps_t();
  mps_init(ctx, m, n);
  size_t off = 0;
  for (int k = 0; k < n; ++k) {
    if (ranks[k + 1] < 1) {
      mps_free(m);
      delete m;
      return fail(ctx, VP_EINVAL, "mps_create_cores: bad rank");
    }
    m->r[k + 1] = ranks[k + 1];
    const size_t e = core_elems(m, k);
    int s = reserve(ctx, m->core[k], e);
    if (s == VP_OK) {
      cudaError_t ce = cudaMemcpyAsync(m->core[k].p, cores + off, e * sizeof(double), cudaMemcpyHostToDevice,
                                       ctx->stream);
      if (ce != cudaSuccess) s = cuda_fail(ctx, ce, "mps_create_cores");
    }
    if (s != VP_OK) {
      mps_free(m);
      delete m;
      return s;
    }
    off += e;
  }
  cudaStreamSynchronize(ctx->stream);
  *out = m;
  return VP_OK;
}

int mps_destroy(mps_t* m) {
  if (!m) return VP_EINVAL;
  mps_free(m);
  delete m;
  return VP_OK;
}

int mps_num_sites(const mps_t* m) { return m ? m->n : -1; }

int mps_bonds(const mps_t* m, int* out) {
  if (!m || !out) return VP_EINVAL;
  for (int k = 0; k <= m->n; ++k) out[k] = m->r[k];
  return VP_OK;
}

int mps_get_cores(vp_ctx* ctx, const mps_t* m, double* host, size_t capacity) {
  if (!ctx || !m || !host) return VP_EINVAL;
  size_t off = 0;
  for (int k = 0; k < m->n; ++k) {
    const size_t e = core_elems(m, k);
    if (off + e > capacity) return fail(ctx, VP_ECAPACITY, "mps_get_cores: buffer too small");
    VP_CUDA(ctx, cudaMemcpyAsync(host + off, m->core[k].p, e * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    off += e;
  }
  VP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return VP_OK;
}

int mps_to_dense(vp_ctx* ctx, const mps_t* m, double* host) {
  if (!ctx || !m || !host || m->n > 24) return fail(ctx, VP_EINVAL, "mps_to_dense: bad argument");
  DevBuf d;
  VP_TRY(to_dense_dev(ctx, m, d));
  VP_CUDA(ctx, cudaMemcpyAsync(host, d.p, ((size_t)1 << m->n) * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  VP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  release(ctx, d);
  return VP_OK;
}

int mps_to_grid(vp_ctx* ctx, const mps_t* m, const vp_layout* L, double* host) {
  if (!ctx || !m || !host || !layout_ok(L) || L->nx + L->nv != m->n)
    return fail(ctx, VP_EINVAL, "mps_to_grid: bad argument");
  DevBuf d, g;
  VP_TRY(to_dense_dev(ctx, m, d));
  const size_t N = (size_t)1 << m->n;
  VP_TRY(reserve(ctx, g, N));
  VP_TRY(launch_permute_to_sites(ctx, d.p, L->nx, L->nv, L->mapping, g.p, 1));
  VP_CUDA(ctx, cudaMemcpyAsync(host, g.p, N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  VP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  release(ctx, d);
  release(ctx, g);
  return VP_OK;
}

// ------------------------------------------------------------------- MPO
static int mpo_from_chain(vp_ctx* ctx, const Chain& c, mpo_t** out) {
  mpo_t* m = new mpo_t();
  m->ctx = ctx;
  m->n = (int)c.core.size();
  m->w = c.w;
  m->core.assign(m->n, DevBuf{});
  for (int k = 0; k < m->n; ++k) {
    int s = reserve(ctx, m->core[k], c.core[k].size());
    if (s == VP_OK) {
      cudaError_t e = cudaMemcpyAsync(m->core[k].p, c.core[k].data(), c.core[k].size() * sizeof(double),
                                      cudaMemcpyHostToDevice, ctx->stream);
      if (e != cudaSuccess) s = cuda_fail(ctx, e, "mpo upload");
    }
    if (s != VP_OK) {
      for (auto& b : m->core) release(ctx, b);
      delete m;
      return s;
    }
  }
  VP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  *out = m;
  return VP_OK;
}

}  // extern "C"
namespace vp {
double grid_dx(const vp_layout* L) { return (L->xmax - L->xmin) / (double)(1 << L->nx); }
double grid_dv(const vp_layout* L) { return (L->vmax - L->vmin) / (double)((1 << L->nv) - 1); }
}  // namespace vp
extern "C" {

int mpo_create_vp(vp_ctx* ctx, const vp_layout* L, int kind, mpo_t** out) {
  if (!ctx || !out || !layout_ok(L)) return fail(ctx, VP_EINVAL, "mpo_create_vp: bad argument");
  const std::vector<int> dims = site_dims(L);
  const double dx = grid_dx(L), dv = grid_dv(L);
  auto ox = [&](Chain ch) { return xdesc(L) ? reverse_chain(ch) : ch; };
  auto ov = [&](Chain ch) { return vdesc(L) ? reverse_chain(ch) : ch; };
  Chain c;
  switch (kind) {
    case VP_MPO_DX_CENTERED:
      c = place2(ox(stencil_chain(L->nx, {{0.0, -0.5 / dx, 0.0, 0.5 / dx, 0.0}}, true)), identity_chain(L->nv), dims);
      break;
    case VP_MPO_DX_FORWARD:
      c = place2(ox(stencil_chain(L->nx, {{0.0, 0.0, -1.5 / dx, 2.0 / dx, -0.5 / dx}}, true)),
                 identity_chain(L->nv), dims);
      break;
    case VP_MPO_DX_BACKWARD:
      c = place2(ox(stencil_chain(L->nx, {{0.5 / dx, -2.0 / dx, 1.5 / dx, 0.0, 0.0}}, true)),
                 identity_chain(L->nv), dims);
      break;
    case VP_MPO_DV_ZERO_GRAD:
      c = place2(identity_chain(L->nx), ov(zero_gradient_chain(L->nv, dv)), dims);
      break;
    case VP_MPO_DXX: {
      const double s = 1.0 / (dx * dx);
      c = place2(ox(stencil_chain(L->nx, {{0.0, s, -2.0 * s, s, 0.0}}, true)), identity_chain(L->nv), dims);
      break;
    }
    case VP_MPO_ADVECTION:
      c = upwind_operator(L->nx, L->nv, dims, dx, L->vmin, dv, xdesc(L), vdesc(L));
      break;
    default:
      return fail(ctx, VP_EINVAL, "mpo_create_vp: unknown kind");
  }
  return mpo_from_chain(ctx, c, out);
}

int mpo_create_cores(vp_ctx* ctx, int n, const int* bonds, const double* cores, mpo_t** out) {
  if (!ctx || n < 1 || !bonds || !cores || !out || bonds[0] != 1 || bonds[n] != 1)
    return fail(ctx, VP_EINVAL, "mpo_create_cores: bad argument");
  Chain c;
  c.alloc(std::vector<int>(bonds, bonds + n + 1));
  size_t off = 0;
  for (int k = 0; k < n; ++k) {
    std::memcpy(c.core[k].data(), cores + off, c.core[k].size() * sizeof(double));
    off += c.core[k].size();
  }
  return mpo_from_chain(ctx, c, out);
}

int mpo_destroy(mpo_t* m) {
  if (!m) return VP_EINVAL;
  for (auto& b : m->core) release(m->ctx, b);
  delete m;
  return VP_OK;
}

int mpo_num_sites(const mpo_t* m) { return m ? m->n : -1; }

int mpo_bonds(const mpo_t* m, int* out) {
  if (!m || !out) return VP_EINVAL;
  for (int k = 0; k <= m->n; ++k) out[k] = m->w[k];
  return VP_OK;
}

int mpo_to_dense(vp_ctx* ctx, const mpo_t* m, double* host) {
  if (!ctx || !m || !host || m->n > 12) return fail(ctx, VP_EINVAL, "mpo_to_dense: bad argument");
  DevBuf a, b;
  // T[o_prev][i_prev][w] starting from the first core (1,2,2,w1)
  VP_TRY(reserve(ctx, a, (size_t)4 * m->w[1]));
  VP_TRY(launch_copy(ctx, m->core[0].p, a.p, (size_t)4 * m->w[1]));
  int rows = 2;
  for (int k = 1; k < m->n; ++k) {
    const size_t no = (size_t)rows * 2;
    VP_TRY(reserve(ctx, b, no * no * m->w[k + 1]));
    VP_TRY(launch_mpo_dense_step(ctx, a.p, rows, rows, m->w[k], m->core[k].p, m->w[k + 1], b.p));
    std::swap(a, b);
    rows *= 2;
  }
  const size_t N = (size_t)1 << m->n;
  VP_CUDA(ctx, cudaMemcpyAsync(host, a.p, N * N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  VP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  release(ctx, a);
  release(ctx, b);
  return VP_OK;
}

// ------------------------------------------------------------ operations
static int site_sum_mps(vp_ctx* ctx, double alpha, const mps_t* a, double beta, const mpo_t* B, const mps_t* b,
                        mps_t* out) {
  const int n = b->n;
  if ((a && a->n != n) || (B && B->n != n)) return fail(ctx, VP_EINVAL, "site counts differ");
  std::vector<int> r(n + 1, 1);
  for (int k = 1; k < n; ++k) r[k] = (a ? a->r[k] : 0) + b->r[k] * (B ? B->w[k] : 1);
  if (out->n != n) {
    mps_free(out);
    mps_init(ctx, out, n);
  }
  for (int k = 0; k < n; ++k) {
    SiteSum s{};
    s.a = a ? a->core[k].p : nullptr;
    s.al = a ? a->r[k] : 0;
    s.ar = a ? a->r[k + 1] : 0;
    s.b = b->core[k].p;
    s.bl = b->r[k];
    s.br = b->r[k + 1];
    s.B = B ? B->core[k].p : nullptr;
    s.wl = B ? B->w[k] : 1;
    s.wr = B ? B->w[k + 1] : 1;
    s.alpha = (k == 0) ? alpha : 1.0;
    s.beta = (k == 0) ? beta : 1.0;
    s.first = (k == 0);
    s.last = (k == n - 1);
    VP_TRY(reserve(ctx, out->core[k], (size_t)r[k] * 2 * r[k + 1]));
    prof_begin(ctx, VP_K_APPLY);
    VP_TRY(launch_site_sum(ctx, s, out->core[k].p, r[k], r[k + 1]));
    const double bytes = 8.0 * ((double)r[k] * 2 * r[k + 1] + (a ? (double)s.al * 2 * s.ar : 0.0) +
                                (double)s.bl * 2 * s.br + (B ? (double)s.wl * 4 * s.wr : 0.0));
    prof_end(ctx, VP_K_APPLY, bytes);
  }
  out->r = r;
  return VP_OK;
}

int mps_apply_mpo(vp_ctx* ctx, const mpo_t* mpo, const mps_t* in, mps_t* out) {
  if (!ctx || !mpo || !in || !out || in == out) return fail(ctx, VP_EINVAL, "mps_apply_mpo: bad argument");
  VP_TRY(site_sum_mps(ctx, 0.0, nullptr, 1.0, mpo, in, out));
  return sync_status(ctx);
}

int mps_axpby(vp_ctx* ctx, double a, const mps_t* x, double b, const mps_t* y, mps_t* out) {
  if (!ctx || !x || !y || !out || out == x || out == y) return fail(ctx, VP_EINVAL, "mps_axpby: bad argument");
  VP_TRY(site_sum_mps(ctx, a, x, b, nullptr, y, out));
  return sync_status(ctx);
}

int mps_compress_modified(vp_ctx* ctx, mps_t* m, int split, int chi, double tol, double* errs) {
  if (!ctx || !m || chi < 1 || tol < 0 || split < 1 || split >= m->n)
    return fail(ctx, VP_EINVAL, "mps_compress_modified: bad argument");
  std::vector<double> e(std::max(1, m->n - 1), 0.0);
  VP_TRY(compress_modified(ctx, m, split, chi, tol, e.data()));
  VP_TRY(sync_status(ctx));
  if (errs)
    for (int k = 0; k + 1 < m->n; ++k) errs[k] = e[k];
  return VP_OK;
}

int mps_compress(vp_ctx* ctx, mps_t* m, int chi, double tol, double* errs) {
  if (!ctx || !m || chi < 1 || tol < 0) return fail(ctx, VP_EINVAL, "mps_compress: bad argument");
  std::vector<double> e(std::max(1, m->n - 1), 0.0);
  VP_TRY(compress(ctx, m, chi, tol, e.data()));
  VP_TRY(sync_status(ctx));
  if (errs)
    for (int k = 0; k + 1 < m->n; ++k) errs[k] = e[k];
  return VP_OK;
}

int mps_compression_error(vp_ctx* ctx, const mps_t* f, int nchi, const int* chi, double tol, double* rms_out) {
  if (!ctx || !f || nchi < 1 || !chi || !rms_out || tol < 0 || f->n > 24)
    return fail(ctx, VP_EINVAL, "mps_compression_error: bad argument");
  for (int i = 0; i < nchi; ++i)
    if (chi[i] < 1) return fail(ctx, VP_EINVAL, "mps_compression_error: chi < 1");
  const size_t N = (size_t)1 << f->n;
  DevBuf full, part, scratch;
  VP_TRY(to_dense_dev(ctx, f, full));
  VP_TRY(reserve(ctx, scratch, 1024 + 64));
  int st = VP_OK;
  for (int i = 0; i < nchi && st == VP_OK; ++i) {
    mps_t c;
    mps_init(ctx, &c, 0);
    st = mps_copy(ctx, f, &c);
    if (st == VP_OK) st = compress(ctx, &c, chi[i], tol, nullptr);
    if (st == VP_OK) st = to_dense_dev(ctx, &c, part);
    if (st == VP_OK) st = launch_sqdiff(ctx, full.p, part.p, N, scratch.p, scratch.p + 1024 + i % 64);
    if (st == VP_OK && cudaMemcpyAsync(rms_out + i, scratch.p + 1024 + i % 64, sizeof(double), cudaMemcpyDeviceToHost,
                                       ctx->stream) != cudaSuccess)
      st = fail(ctx, VP_ECUDA, "mps_compression_error: copy failed");
    if (st == VP_OK) st = sync_status(ctx);
    mps_free(&c);
    if (st == VP_OK) rms_out[i] = std::sqrt(rms_out[i] / (double)N);
  }
  release(ctx, full);
  release(ctx, part);
  release(ctx, scratch);
  return st;
}

int vp_density(vp_ctx* ctx, const vp_layout* L, const mps_t* f, double* rho_dev) {
  if (!ctx || !f || !rho_dev || !layout_ok(L) || L->nx + L->nv != f->n)
    return fail(ctx, VP_EINVAL, "vp_density: bad argument");
  VP_TRY(density(ctx, L, f, rho_dev));
  return sync_status(ctx);
}

int vp_gemm(vp_ctx* ctx, int precision, int M, int N, int K, double alpha, const double* A, int lda,
            const double* B, int ldb, double* C, int ldc) {
  if (!ctx || M < 0 || N < 0 || K < 0 || (M > 0 && N > 0 && (!C || ldc < N)) ||
      (M > 0 && N > 0 && K > 0 && (!A || !B || lda < K || ldb < N)) || precision < VP_PREC_FP64 ||
      precision > VP_PREC_TF32X3)
    return fail(ctx, VP_EINVAL, "vp_gemm: bad argument");
  const int p0 = ctx->precision;
  ctx->precision = precision;
  const int st = launch_gemm(ctx, M, N, K, alpha, A, lda, B, ldb, C, ldc);
  ctx->precision = p0;
  VP_TRY(st);
  return sync_status(ctx);
}

int vp_poisson(vp_ctx* ctx, const double* rho, int nx, double dx, double* E, double* we_host) {
  if (!ctx || !rho || !E || nx < 1 || nx > 14 || !(dx > 0)) return fail(ctx, VP_EINVAL, "vp_poisson: bad argument");
  VP_TRY(launch_poisson(ctx, rho, 1 << nx, dx, E, ctx->d_smalld + 8));
  VP_CUDA(ctx, cudaMemcpyAsync(ctx->h_smalld + 8, ctx->d_smalld + 8, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                               ctx->stream));
  VP_TRY(sync_status(ctx));
  if (we_host) *we_host = ctx->h_smalld[8];
  return VP_OK;
}

}  // extern "C"

// ====================================================================== stepper

namespace vp {

// Assemble L(E) = U + diag(E) (x) D_v from the current field MPS.
static int assemble_operator(vp_sim* s, bool with_upwind = true, mpo_t* dst = nullptr) {
  vp_ctx* ctx = s->ctx;
  mpo_t& L = dst ? *dst : s->L;
  const int n = (int)s->dims.size();
  const mps_t& em = s->em;
  // bonds of the placed field term: E channel x D_v channel
  std::vector<int> tw(n + 1);
  int px = 0, pv = 0;
  tw[0] = 1;
  for (int k = 0; k < n; ++k) {
    if (s->dims[k] == 0) ++px; else ++pv;
    tw[k + 1] = em.r[px] * s->Dv.w[pv];
  }
  std::vector<int> w(n + 1), uw(n + 1, 0);
  if (with_upwind) uw = s->U.w;
  w[0] = w[n] = 1;
  for (int k = 1; k < n; ++k) w[k] = uw[k] + tw[k];
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
    VP_TRY(launch_assemble_site(ctx, s->Ud[k].p, with_upwind ? s->U.w[k] : 0, with_upwind ? s->U.w[k + 1] : 0, e,
                                k == 0, k == n - 1, L.core[k].p, w[k], w[k + 1]));
  }
  return VP_OK;
}

// E (device, Nx) as an MPS in the site order of the x bits (tolerance
// e_tol, cap e_chi) -> L(E).
static int field_operator(vp_sim* s, const double* E) {
  vp_ctx* ctx = s->ctx;
  const int Nx = 1 << s->lay.nx;
  mps_free(&s->em);
  const double* Ev = E;
  if (xdesc(&s->lay)) {
    VP_TRY(reserve(ctx, s->evec, (size_t)Nx));
    VP_TRY(launch_permute_to_sites(ctx, E, s->lay.nx, 0, VP_SEQ_S2, s->evec.p, 0));
    Ev = s->evec.p;
  }
  const int g0 = ctx->grouped;  // the field MPS holds x bits only: no pairs
  ctx->grouped = 0;
  const int st = from_vector(ctx, &s->em, s->lay.nx, Ev, s->cfg.e_chi > 0 ? s->cfg.e_chi : 1 << 30, s->cfg.e_tol);
  ctx->grouped = g0;
  VP_TRY(st);
  return assemble_operator(s);
}

// Field of a stage: rho -> E -> E as an MPS (tolerance e_tol) -> L(E).
static int stage_operator(vp_sim* s, const mps_t* f, double* we_mass) {
  vp_ctx* ctx = s->ctx;
  const int Nx = 1 << s->lay.nx;
  VP_TRY(density(ctx, &s->lay, f, s->rho.p));
  VP_TRY(launch_poisson(ctx, s->rho.p, Nx, grid_dx(&s->lay), s->E.p, ctx->d_smalld + 8));
  if (we_mass)
    VP_CUDA(ctx, cudaMemcpyAsync(we_mass, ctx->d_smalld + 8, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  return field_operator(s, s->E.p);
}

// Compression levels C2..C5 (and a capped field bond): one stream, the
// schedule spelled out in vp_config.level.
static int sim_step_levels(vp_sim* s, vp_record* rec) {
  vp_ctx* ctx = s->ctx;
  static const double A[3] = {0.5, 0.5, 1.0};
  static const double B[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  static const double Wt[4] = {1.0, 2.0, 2.0, 1.0};
  const int level = std::max(1, s->cfg.level), chi = s->cfg.chi, big = 1 << 30;
  const double dt = s->cfg.dt, tol = s->cfg.tol;
  const mps_t* fi = &s->f;
  const mps_t* acc = &s->f;
  std::vector<double> errs(s->f.n, 0.0);
  g_flops = &s->flops;
  mpo_t Uview;
  Uview.ctx = ctx;
  Uview.n = (int)s->dims.size();
  Uview.w = s->U.w;
  for (int i = 0; i < 4; ++i) {
    VP_TRY(stage_operator(s, fi, i == 0 ? s->ctx->h_smalld + 16 : nullptr));
    if (level >= 5) {
      Uview.core = s->Ud;
      VP_TRY(site_sum_mps(ctx, 0.0, nullptr, 1.0, &Uview, fi, &s->ku));
      Uview.core.clear();
      VP_TRY(compress(ctx, &s->ku, chi, tol, nullptr));
      VP_TRY(assemble_operator(s, false, &s->LT));
      VP_TRY(site_sum_mps(ctx, 0.0, nullptr, 1.0, &s->LT, fi, &s->kt));
      VP_TRY(compress(ctx, &s->kt, chi, tol, nullptr));
      VP_TRY(site_sum_mps(ctx, 1.0, &s->ku, 1.0, nullptr, &s->kt, &s->kd));
      VP_TRY(compress(ctx, &s->kd, chi, tol, nullptr));
    } else {
      VP_TRY(site_sum_mps(ctx, 0.0, nullptr, 1.0, &s->L, fi, &s->kd));
      if (level >= 4) VP_TRY(compress(ctx, &s->kd, chi, tol, nullptr));
    }
    if (level >= 3) {
      if (i == 0) {
        VP_TRY(mps_copy(ctx, &s->kd, &s->acc));
      } else {
        VP_TRY(site_sum_mps(ctx, 1.0, &s->acc, Wt[i], nullptr, &s->kd, &s->wa));
        VP_TRY(compress(ctx, &s->wa, chi, tol, nullptr));
        std::swap(s->acc, s->wa);
      }
    } else if (i < 3) {
      VP_TRY(site_sum_mps(ctx, 1.0, acc, B[i] * dt, nullptr, &s->kd, &s->wa));
      VP_TRY(compress(ctx, &s->wa, big, tol, nullptr));
      std::swap(s->acc, s->wa);
      acc = &s->acc;
    }
    if (i < 3) {
      VP_TRY(site_sum_mps(ctx, 1.0, &s->f, A[i] * dt, nullptr, &s->kd, &s->wb));
      VP_TRY(compress(ctx, &s->wb, level >= 2 ? chi : big, tol, nullptr));
      std::swap(s->fi, s->wb);
      fi = &s->fi;
    }
  }
  if (level >= 3)
    VP_TRY(site_sum_mps(ctx, 1.0, &s->f, dt / 6.0, nullptr, &s->acc, &s->wa));
  else
    VP_TRY(site_sum_mps(ctx, 1.0, acc, B[3] * dt, nullptr, &s->kd, &s->wa));
  s->entropy.assign(std::max(1, s->f.n - 1), 0.0);
  g_entropy = s->entropy.data();
  const int stc = compress(ctx, &s->wa, chi, tol, errs.data());
  g_entropy = nullptr;
  VP_TRY(stc);
  std::swap(s->f, s->wa);
  g_flops = nullptr;
  VP_TRY(sync_status(ctx));
  const double we = s->ctx->h_smalld[16], mass = s->ctx->h_smalld[17];
  if (!std::isfinite(we)) return fail(ctx, VP_ENUMERIC, "non-finite field energy");
  if (rec) {
    rec->t = s->t;
    rec->field_energy = we;
    rec->mass = mass;
    rec->max_bond = *std::max_element(s->f.r.begin(), s->f.r.end());
    rec->trunc_err = errs.empty() ? 0.0 : *std::max_element(errs.begin(), errs.end());
  }
  s->t += dt;
  return VP_OK;
}

static int sim_step_impl(vp_sim* s, vp_record* rec);

// The contraction precision applies to this sim's steps only.
// So does the compression scheme (the modified one cuts first at the x / v
// bond, after the x sites).
// cfg.streams == 0 on an eligible sim: the step runs as a one-member
// lockstep group (the stage's two compressions share every launch), with the
// same arithmetic as the paths below.
static int sim_step_lockstep(vp_sim* s, vp_record* rec) {
  vp_ctx* ctx = s->ctx;
  if (!s->lockstep) {
    VP_TRY(vp_group_create(ctx, 1, &s->lockstep));
    const int st = vp_group_add(s->lockstep, s);
    if (st != VP_OK) {
      vp_group_destroy(s->lockstep);
      s->lockstep = nullptr;
      return st;
    }
  }
  int mst = VP_OK;
  VP_TRY(vp_group_step(s->lockstep, rec, &mst));
  if (mst == VP_ETIMEOUT) return fail(ctx, mst, "a device-side wait gave up");
  if (mst != VP_OK) return fail(ctx, mst, "NaN or Inf in the field or the singular values, or a Jacobi SVD that did not converge");
  return VP_OK;
}

static int sim_step(vp_sim* s, vp_record* rec) {
  if (s->cfg.streams == 0 && !s->ctxB && lockstep_eligible(s)) return sim_step_lockstep(s, rec);
  const int p0 = s->ctx->precision, m0 = s->ctx->modified_split, g0 = s->ctx->grouped;
  const int split = s->cfg.compression == VP_COMPRESS_MODIFIED ? s->lay.nx : 0;
  s->ctx->precision = s->cfg.precision;
  s->ctx->modified_split = split;
  s->ctx->grouped = grouped(&s->lay) ? 1 : 0;
  if (s->ctxB) {
    s->ctxB->precision = s->cfg.precision;
    s->ctxB->modified_split = split;
    s->ctxB->grouped = s->ctx->grouped;
  }
  const int st = s->cfg.level > 1 ? sim_step_levels(s, rec) : sim_step_impl(s, rec);
  s->ctx->precision = p0;
  s->ctx->modified_split = m0;
  s->ctx->grouped = g0;
  return st;
}

// Stage i of RK4-C1 once the stage operator L is assembled: for i < 3
// acc <- C_tol(acc + B_i dt L f_i) and f_{i+1} <- C_tol(f + A_i dt L f_i)
// (concurrently on the second stream when there is one); for i = 3
// f <- C_chi(acc + B_3 dt L f_3), its per-bond errors in errs.
static int c1_stage(vp_sim* s, int i, const mps_t*& fi, const mps_t*& acc, double* errs) {
  vp_ctx* ctx = s->ctx;
  static const double A[3] = {0.5, 0.5, 1.0};
  static const double B[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  const double dt = s->cfg.dt;
  if (i < 3 && s->ctxB) {
    // The two tolerance compressions of a stage are independent: acc_i on
    // this context's stream, f_{i+1} on the second stream from a second
    // host thread.  Each MPS keeps its buffers on the context that
    // compresses it (acc, wa, f: first; fi, wb: second).
    vp_ctx* cb = s->ctxB;
    VP_CUDA(ctx, cudaEventRecord(s->evA, ctx->stream));
    VP_CUDA(ctx, cudaStreamWaitEvent(cb->stream, s->evA, 0));
    VP_TRY(site_sum_mps(ctx, 1.0, acc, B[i] * dt, &s->L, fi, &s->wa));
    VP_TRY(site_sum_mps(cb, 1.0, &s->f, A[i] * dt, &s->L, fi, &s->wb));
    const int cap0 = ctx->coop_cap;
    ctx->coop_cap = cb->coop_cap = std::max(2, ctx->num_sms / (2 * s->coop_div));
    int stB = VP_OK;
    Flops fB;
    const bool prof = ctx->prof_on;
    std::thread worker([&] {
      cb->prof_on = prof;
      g_flops = &fB;
      stB = compress(cb, &s->wb, 1 << 30, s->cfg.tol, nullptr);
      g_flops = nullptr;
    });
    const int stA = compress(ctx, &s->wa, 1 << 30, s->cfg.tol, nullptr);
    worker.join();
    ctx->coop_cap = cap0;
    if (stA != VP_OK) return stA;
    if (stB != VP_OK) return fail(ctx, stB, cb->err);
    VP_CUDA(ctx, cudaEventRecord(s->evB, cb->stream));
    VP_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, s->evB, 0));
    s->flops.qr += fB.qr;
    s->flops.formq += fB.formq;
    s->flops.gemm += fB.gemm;
    s->flops.jacobi += fB.jacobi;
    std::swap(s->acc, s->wa);
    std::swap(s->fi, s->wb);
    acc = &s->acc;
    fi = &s->fi;
  } else if (i < 3) {
    VP_TRY(site_sum_mps(ctx, 1.0, acc, B[i] * dt, &s->L, fi, &s->wa));
    VP_TRY(site_sum_mps(ctx, 1.0, &s->f, A[i] * dt, &s->L, fi, &s->wb));
    VP_TRY(compress(ctx, &s->wa, 1 << 30, s->cfg.tol, nullptr));
    VP_TRY(compress(ctx, &s->wb, 1 << 30, s->cfg.tol, nullptr));
    std::swap(s->acc, s->wa);
    std::swap(s->fi, s->wb);
    acc = &s->acc;
    fi = &s->fi;
  } else {
    VP_TRY(site_sum_mps(ctx, 1.0, acc, B[3] * dt, &s->L, fi, &s->wa));
    s->entropy.assign(std::max(1, s->f.n - 1), 0.0);
    g_entropy = s->entropy.data();
    const int stc = compress(ctx, &s->wa, s->cfg.chi, s->cfg.tol, errs);
    g_entropy = nullptr;
    VP_TRY(stc);
    std::swap(s->f, s->wa);
  }
  return VP_OK;
}

static int sim_step_impl(vp_sim* s, vp_record* rec) {
  vp_ctx* ctx = s->ctx;
  const mps_t* fi = &s->f;
  const mps_t* acc = &s->f;
  double wm[2] = {0, 0};
  std::vector<double> errs(s->f.n, 0.0);
  g_flops = &s->flops;
  for (int i = 0; i < 4; ++i) {
    VP_TRY(stage_operator(s, fi, i == 0 ? s->ctx->h_smalld + 16 : nullptr));
    VP_TRY(c1_stage(s, i, fi, acc, errs.data()));
  }
  g_flops = nullptr;
  VP_TRY(sync_status(ctx));
  wm[0] = s->ctx->h_smalld[16];
  wm[1] = s->ctx->h_smalld[17];
  if (!std::isfinite(wm[0])) return fail(ctx, VP_ENUMERIC, "non-finite field energy");
  if (rec) {
    rec->t = s->t;
    rec->field_energy = wm[0];
    rec->mass = wm[1];
    rec->max_bond = *std::max_element(s->f.r.begin(), s->f.r.end());
    rec->trunc_err = errs.empty() ? 0.0 : *std::max_element(errs.begin(), errs.end());
  }
  s->t += s->cfg.dt;
  return VP_OK;
}

static int upload_chain(vp_ctx* ctx, const Chain& c, std::vector<DevBuf>& out) {
  out.assign(c.core.size(), DevBuf{});
  for (size_t k = 0; k < c.core.size(); ++k) {
    VP_TRY(reserve(ctx, out[k], std::max<size_t>(1, c.core[k].size())));
    VP_CUDA(ctx, cudaMemcpyAsync(out[k].p, c.core[k].data(), c.core[k].size() * sizeof(double),
                                 cudaMemcpyHostToDevice, ctx->stream));
  }
  VP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return VP_OK;
}

static void sim_free(vp_sim* s) {
  vp_ctx* ctx = s->ctx;
  if (s->lockstep) {
    vp_group_destroy(s->lockstep);
    s->lockstep = nullptr;
  }
  if (s->ctxB) {
    cudaStreamSynchronize(s->ctxB->stream);
    cudaStreamSynchronize(ctx->stream);
    for (mps_t* m : {&s->fi, &s->wb}) {
      m->ctx = s->ctxB;  // these buffers belong to the second context
      mps_free(m);
    }
    auto& ch = ctx->children;
    ch.erase(std::remove(ch.begin(), ch.end(), s->ctxB), ch.end());
    vp_ctx_destroy(s->ctxB);
    s->ctxB = nullptr;
  }
  if (s->evA) cudaEventDestroy(s->evA);
  if (s->evB) cudaEventDestroy(s->evB);
  for (mps_t* m : {&s->f, &s->fi, &s->acc, &s->wa, &s->wb, &s->em, &s->kd, &s->ku, &s->kt}) mps_free(m);
  for (auto& b : s->LT.core) release(ctx, b);
  for (auto& b : s->Ud) release(ctx, b);
  for (auto& b : s->Dvd) release(ctx, b);
  for (auto& b : s->L.core) release(ctx, b);
  release(ctx, s->rho);
  release(ctx, s->E);
  release(ctx, s->evec);
}

// A sim of one species: sp == NULL is the electron species against a fixed
// neutralising background; otherwise the field factor -q/m and, for nu > 0,
// the Dougherty term joins the static part of the operator.
static int sim_create(vp_ctx* ctx, const vp_layout* L, const vp_config* cfg, const mps_t* f0, const vp_species* sp,
                      vp_sim** out) {
  if (!ctx || !cfg || !f0 || !out || !layout_ok(L) || L->nx + L->nv != f0->n || cfg->chi < 1 || cfg->tol < 0 ||
      cfg->e_tol < 0 || !(cfg->dt > 0))
    return fail(ctx, VP_EINVAL, "vp_sim_create: bad argument");
  const double dx = grid_dx(L);
  if (std::max(std::fabs(L->vmin), std::fabs(L->vmax)) * cfg->dt / dx > 0.6963)
    return fail(ctx, VP_ECFL, "dt above the RK4 upwind stability limit");
  vp_sim* s = new vp_sim();
  s->ctx = ctx;
  s->lay = *L;
  s->cfg = *cfg;
  s->dims = site_dims(L);
  for (mps_t* m : {&s->f, &s->fi, &s->acc, &s->wa, &s->wb, &s->em, &s->kd, &s->ku, &s->kt}) mps_init(ctx, m, 0);
  int st = mps_copy(ctx, f0, &s->f);
  if (st == VP_OK) {
    s->U = upwind_operator(L->nx, L->nv, s->dims, dx, L->vmin, grid_dv(L), xdesc(L), vdesc(L));
    if (sp) {
      s->ecoef = -sp->q / sp->m;
      if (sp->nu > 0.0) {
        Chain cv = collision_chain(L->nv, L->vmin, grid_dv(L), sp->nu, sp->u, sp->vth);
        if (vdesc(L)) cv = reverse_chain(cv);
        // the summed chain carries redundant channels (bond 15 on the v
        // sites for a numerical rank of 6): reduce it once, exactly
        s->U = reduce_chain(chain_sum(s->U, place2(identity_chain(L->nx), cv, s->dims)), 1e-13);
      }
    }
    s->Dv = zero_gradient_chain(L->nv, grid_dv(L));
    if (vdesc(L)) s->Dv = reverse_chain(s->Dv);
    st = upload_chain(ctx, s->U, s->Ud);
  }
  if (st == VP_OK) st = upload_chain(ctx, s->Dv, s->Dvd);
  if (st == VP_OK) st = reserve(ctx, s->rho, (size_t)1 << L->nx);
  if (st == VP_OK) st = reserve(ctx, s->E, (size_t)1 << L->nx);
  if (cfg->level < 0 || cfg->level > 5 || cfg->e_chi < 0 || cfg->precision < VP_PREC_FP64 || cfg->precision > VP_PREC_TF32X3)
    st = fail(ctx, VP_EINVAL, "vp_sim_create: bad level/e_chi/precision");
  if (st == VP_OK && (cfg->compression < VP_COMPRESS_SWEEPS || cfg->compression > VP_COMPRESS_MODIFIED ||
                      (cfg->compression == VP_COMPRESS_MODIFIED && (interleaved(L) || L->nx < 1 || L->nv < 1))))
    st = fail(ctx, VP_EINVAL, "vp_sim_create: the modified compression needs a sequential ordering");
  // streams 2, or 0 where the lockstep path does not apply: the second stream
  const bool lock = cfg->streams == 0 && !sp && lockstep_eligible(s);
  if (st == VP_OK && cfg->streams != 1 && cfg->level <= 1 && !lock) {
    s->ctxB = ctx_child(ctx);
    if (s->ctxB) {
      s->fi.ctx = s->wb.ctx = s->ctxB;
      if (cudaEventCreateWithFlags(&s->evA, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&s->evB, cudaEventDisableTiming) != cudaSuccess)
        st = fail(ctx, VP_ECUDA, "vp_sim_create: event creation failed");
    }
  }
  if (st == VP_OK) st = sync_status(ctx);
  if (st != VP_OK) {
    sim_free(s);
    delete s;
    return st;
  }
  *out = s;
  return VP_OK;
}

}  // namespace vp

extern "C" {

int vp_sim_create(vp_ctx* ctx, const vp_layout* L, const vp_config* cfg, const mps_t* f0, vp_sim** out) {
  return sim_create(ctx, L, cfg, f0, nullptr, out);
}

int vp_sim_destroy(vp_sim* s) {
  if (!s) return VP_EINVAL;
  sim_free(s);
  delete s;
  return VP_OK;
}

int vp_step(vp_sim* s, int nsteps, vp_record* records) {
  if (!s || nsteps < 0) return VP_EINVAL;
  for (int i = 0; i < nsteps; ++i) VP_TRY(sim_step(s, records ? records + i : nullptr));
  return VP_OK;
}

const mps_t* vp_sim_state(const vp_sim* s) { return s ? &s->f : nullptr; }

int vp_sim_entropy(const vp_sim* s, double* out) {
  if (!s || !out) return VP_EINVAL;
  for (int k = 0; k + 1 < s->f.n; ++k) out[k] = k < (int)s->entropy.size() ? s->entropy[k] : 0.0;
  return VP_OK;
}

double vp_sim_flops(const vp_sim* s) {
  return s ? s->flops.qr + s->flops.formq + s->flops.gemm + s->flops.jacobi : 0.0;
}

int vp_run(vp_ctx* ctx, const vp_layout* L, const vp_config* cfg, const double* f0, int nsteps, double* fT,
           vp_record* records) {
  if (!ctx || !cfg || !f0 || nsteps < 0) return fail(ctx, VP_EINVAL, "vp_run: bad argument");
  mps_t* m = nullptr;
  VP_TRY(mps_create(ctx, L, f0, 0, cfg->chi, cfg->tol, &m));
  vp_sim* s = nullptr;
  int st = vp_sim_create(ctx, L, cfg, m, &s);
  mps_destroy(m);
  if (st != VP_OK) return st;
  st = vp_step(s, nsteps, records);
  if (st == VP_OK && fT) st = mps_to_grid(ctx, &s->f, L, fT);
  vp_sim_destroy(s);
  return st;
}

}  // extern "C"

// ================================================================ several species
struct vp_multi {
  vp_ctx* ctx = nullptr;
  std::vector<vp_sim*> sp;
  std::vector<vp_species> par;
  std::vector<vp_ctx*> sctx;       // context of each species' sim (children of ctx when ns > 1)
  std::vector<cudaEvent_t> sev;    // per species: its stream has finished a stage
  cudaEvent_t mev = nullptr;       // the main stream has the stage field
  vp_config cfg{};
  DevBuf net, E, Es;
  double t = 0.0;
};

namespace vp {

// One RK4-C1 step of all species in lockstep: per stage every species'
// density, one Poisson solve for the net density, then each species' field
// operator (E scaled by -q/m) and its C1 stage update.
static int multi_step_impl(vp_multi* M, vp_record* rec) {
  vp_ctx* ctx = M->ctx;
  const int ns = (int)M->sp.size();
  const vp_layout& L0 = M->sp[0]->lay;
  const int Nx = 1 << L0.nx;
  const double dx = grid_dx(&L0);
  std::vector<const mps_t*> fi(ns), acc(ns);
  std::vector<std::vector<double>> errs(ns);
  SpeciesRho sr{};
  sr.ns = ns;
  for (int s = 0; s < ns; ++s) {
    fi[s] = acc[s] = &M->sp[s]->f;
    errs[s].assign(M->sp[s]->f.n, 0.0);
    sr.rho[s] = M->sp[s]->rho.p;
    sr.w[s] = -M->par[s].q;
  }
  const bool par = ns > 1 && M->sctx[0] != ctx;  // species on their own streams, one host thread each
  for (int i = 0; i < 4; ++i) {
    if (par)  // the stage states were written on the species' streams
      for (int s = 0; s < ns; ++s) {
        VP_CUDA(ctx, cudaEventRecord(M->sev[s], M->sctx[s]->stream));
        VP_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, M->sev[s], 0));
      }
    for (int s = 0; s < ns; ++s) VP_TRY(density(ctx, &M->sp[s]->lay, fi[s], M->sp[s]->rho.p));
    VP_TRY(launch_species_net(ctx, sr, Nx, dx, M->net.p, ctx->d_smalld + 32));
    VP_TRY(launch_poisson(ctx, M->net.p, Nx, dx, M->E.p, ctx->d_smalld + 8));
    if (i == 0) {
      VP_CUDA(ctx, cudaMemcpyAsync(ctx->h_smalld + 24, ctx->d_smalld + 8, sizeof(double), cudaMemcpyDeviceToHost,
                                   ctx->stream));
      VP_CUDA(ctx, cudaMemcpyAsync(ctx->h_smalld + 32, ctx->d_smalld + 32, ns * sizeof(double),
                                   cudaMemcpyDeviceToHost, ctx->stream));
    }
    if (par) VP_CUDA(ctx, cudaEventRecord(M->mev, ctx->stream));
    // one species' stage: its field operator (E scaled by -q/m) and C1 update
    auto species_stage = [&](int s) -> int {
      vp_sim* sp = M->sp[s];
      vp_ctx* cs = sp->ctx;
      const double* Ev = M->E.p;
      if (par) {
        VP_CUDA(cs, cudaStreamWaitEvent(cs->stream, M->mev, 0));
        VP_TRY(launch_copy(cs, M->E.p, sp->E.p, (size_t)Nx));
        if (sp->ecoef != 1.0) VP_TRY(launch_scale(cs, sp->E.p, (size_t)Nx, sp->ecoef));
        Ev = sp->E.p;
      } else if (sp->ecoef != 1.0) {
        VP_TRY(launch_copy(cs, M->E.p, M->Es.p, (size_t)Nx));
        VP_TRY(launch_scale(cs, M->Es.p, (size_t)Nx, sp->ecoef));
        Ev = M->Es.p;
      }
      VP_TRY(field_operator(sp, Ev));
      g_flops = &sp->flops;
      const int g0 = cs->grouped;
      cs->grouped = grouped(&sp->lay) ? 1 : 0;
      if (sp->ctxB) sp->ctxB->grouped = cs->grouped;
      const int st = c1_stage(sp, i, fi[s], acc[s], errs[s].data());
      cs->grouped = g0;
      g_flops = nullptr;
      return st;
    };
    if (par) {
      std::vector<int> st(ns, VP_OK);
      std::vector<std::thread> th;
      for (int s = 1; s < ns; ++s) th.emplace_back([&, s] { st[s] = species_stage(s); });
      st[0] = species_stage(0);
      for (auto& t : th) t.join();
      for (int s = 0; s < ns; ++s)
        if (st[s] != VP_OK) return fail(ctx, st[s], M->sctx[s]->err);
    } else {
      for (int s = 0; s < ns; ++s) VP_TRY(species_stage(s));
    }
  }
  if (par)
    for (int s = 0; s < ns; ++s) {
      const int st = sync_status(M->sctx[s]);
      if (st != VP_OK) return fail(ctx, st, M->sctx[s]->err);
    }
  VP_TRY(sync_status(ctx));
  const double we = ctx->h_smalld[24];
  if (!std::isfinite(we)) return fail(ctx, VP_ENUMERIC, "non-finite field energy");
  for (int s = 0; s < ns; ++s) {
    vp_sim* sp = M->sp[s];
    if (rec) {
      rec[s].t = M->t;
      rec[s].field_energy = we;
      rec[s].mass = ctx->h_smalld[32 + s];
      rec[s].max_bond = *std::max_element(sp->f.r.begin(), sp->f.r.end());
      rec[s].trunc_err = errs[s].empty() ? 0.0 : *std::max_element(errs[s].begin(), errs[s].end());
    }
    sp->t += M->cfg.dt;
  }
  M->t += M->cfg.dt;
  return VP_OK;
}

static int multi_step(vp_multi* M, vp_record* rec) {
  vp_ctx* ctx = M->ctx;
  const int p0 = ctx->precision, m0 = ctx->modified_split;
  const int split = M->cfg.compression == VP_COMPRESS_MODIFIED ? M->sp[0]->lay.nx : 0;
  ctx->precision = M->cfg.precision;
  ctx->modified_split = split;
  for (vp_sim* sp : M->sp)
    for (vp_ctx* c : {sp->ctx, sp->ctxB})
      if (c) {
        c->precision = M->cfg.precision;
        c->modified_split = split;
      }
  const int st = multi_step_impl(M, rec);
  ctx->precision = p0;
  ctx->modified_split = m0;
  return st;
}

static void multi_free(vp_multi* M) {
  cudaStreamSynchronize(M->ctx->stream);
  for (vp_sim* s : M->sp) {
    sim_free(s);
    delete s;
  }
  M->sp.clear();
  auto& ch = M->ctx->children;
  for (vp_ctx* c : M->sctx)
    if (c && c != M->ctx) {
      ch.erase(std::remove(ch.begin(), ch.end(), c), ch.end());
      vp_ctx_destroy(c);
    }
  M->sctx.clear();
  for (cudaEvent_t e : M->sev)
    if (e) cudaEventDestroy(e);
  M->sev.clear();
  if (M->mev) cudaEventDestroy(M->mev);
  M->mev = nullptr;
  release(M->ctx, M->net);
  release(M->ctx, M->E);
  release(M->ctx, M->Es);
}

}  // namespace vp

extern "C" {

int vp_multi_create(vp_ctx* ctx, int ns, const vp_layout* layouts, const vp_species* species, const vp_config* cfg,
                    const mps_t* const* f0, vp_multi** out) {
  if (!ctx || ns < 1 || ns > kMaxSpecies || !layouts || !species || !cfg || !f0 || !out || cfg->level > 1)
    return fail(ctx, VP_EINVAL, "vp_multi_create: bad argument");
  for (int s = 0; s < ns; ++s) {
    const vp_layout& L = layouts[s];
    const vp_species& p = species[s];
    if (!layout_ok(&L) || L.nx != layouts[0].nx || L.xmin != layouts[0].xmin || L.xmax != layouts[0].xmax || !f0[s])
      return fail(ctx, VP_EINVAL, "vp_multi_create: every species needs a valid layout on the same x grid");
    if (!(p.m > 0.0) || !std::isfinite(p.q) || !(p.nu >= 0.0) || !std::isfinite(p.u) || (p.nu > 0.0 && !(p.vth > 0.0)))
      return fail(ctx, VP_EINVAL, "vp_multi_create: bad species parameters");
  }
  vp_multi* M = new vp_multi();
  M->ctx = ctx;
  M->cfg = *cfg;
  M->par.assign(species, species + ns);
  int st = VP_OK;
  // with several species, each runs on a child context (own stream) so that
  // their stage updates proceed concurrently; f0 is read on those streams
  VP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (int s = 0; s < ns && st == VP_OK; ++s) {
    vp_ctx* cs = ns > 1 ? ctx_child(ctx) : ctx;
    if (!cs) {
      st = fail(ctx, VP_ENOMEM, "vp_multi_create: no context for a species");
      break;
    }
    M->sctx.push_back(cs);
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      st = fail(ctx, VP_ECUDA, "vp_multi_create: event creation failed");
      break;
    }
    M->sev.push_back(e);
    vp_sim* sim = nullptr;
    st = sim_create(cs, &layouts[s], cfg, f0[s], &species[s], &sim);
    if (st != VP_OK && cs != ctx) st = fail(ctx, st, cs->err);
    if (st == VP_OK) {
      sim->coop_div = ns;
      M->sp.push_back(sim);
    }
  }
  if (st == VP_OK && cudaEventCreateWithFlags(&M->mev, cudaEventDisableTiming) != cudaSuccess)
    st = fail(ctx, VP_ECUDA, "vp_multi_create: event creation failed");
  const size_t Nx = (size_t)1 << layouts[0].nx;
  if (st == VP_OK) st = reserve(ctx, M->net, Nx);
  if (st == VP_OK) st = reserve(ctx, M->E, Nx);
  if (st == VP_OK) st = reserve(ctx, M->Es, Nx);
  if (st != VP_OK) {
    multi_free(M);
    delete M;
    return st;
  }
  *out = M;
  return VP_OK;
}

int vp_multi_destroy(vp_multi* M) {
  if (!M) return VP_EINVAL;
  multi_free(M);
  delete M;
  return VP_OK;
}

int vp_multi_step(vp_multi* M, int nsteps, vp_record* records) {
  if (!M || nsteps < 0) return VP_EINVAL;
  const int ns = (int)M->sp.size();
  for (int n = 0; n < nsteps; ++n) VP_TRY(multi_step(M, records ? records + (size_t)n * ns : nullptr));
  return VP_OK;
}

const mps_t* vp_multi_state(const vp_multi* M, int s) {
  return (M && s >= 0 && s < (int)M->sp.size()) ? &M->sp[s]->f : nullptr;
}

}  // extern "C"

extern "C" int mpo_create_vlasov(vp_ctx* ctx, const vp_layout* L, const double* E_host, double e_tol, mpo_t** out) {
  if (!ctx || !out || !E_host || !layout_ok(L) || e_tol < 0) return fail(ctx, VP_EINVAL, "mpo_create_vlasov: bad argument");
  vp_sim s;
  s.ctx = ctx;
  s.lay = *L;
  s.dims = site_dims(L);
  for (mps_t* m : {&s.f, &s.fi, &s.acc, &s.wa, &s.wb, &s.em}) mps_init(ctx, m, 0);
  s.U = upwind_operator(L->nx, L->nv, s.dims, grid_dx(L), L->vmin, grid_dv(L), xdesc(L), vdesc(L));
  s.Dv = zero_gradient_chain(L->nv, grid_dv(L));
  if (vdesc(L)) s.Dv = reverse_chain(s.Dv);
  int st = upload_chain(ctx, s.U, s.Ud);
  if (st == VP_OK) st = upload_chain(ctx, s.Dv, s.Dvd);
  if (st == VP_OK) st = reserve(ctx, s.E, (size_t)1 << L->nx);
  if (st == VP_OK) {
    cudaError_t e = cudaMemcpyAsync(s.E.p, E_host, sizeof(double) << L->nx, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) st = cuda_fail(ctx, e, "mpo_create_vlasov");
  }
  if (st == VP_OK && xdesc(L)) {
    st = reserve(ctx, s.evec, (size_t)1 << L->nx);
    if (st == VP_OK) st = launch_permute_to_sites(ctx, s.E.p, L->nx, 0, VP_SEQ_S2, s.evec.p, 0);
  }
  if (st == VP_OK) st = from_vector(ctx, &s.em, L->nx, xdesc(L) ? s.evec.p : s.E.p, 1 << 30, e_tol);
  if (st == VP_OK) st = assemble_operator(&s);
  if (st == VP_OK) st = sync_status(ctx);
  if (st == VP_OK) {
    mpo_t* m = new mpo_t();
    m->ctx = ctx;
    m->n = s.L.n;
    m->w = s.L.w;
    m->core = s.L.core;
    s.L.core.clear();
    *out = m;
  }
  sim_free(&s);
  return st;
}
