// Internal declarations shared by the vpmps translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/vpmps.h"

namespace vp {

constexpr int kThreads = 256;      // threads per block of the factorisation kernels
constexpr int kWarps = kThreads / 32;
constexpr long long kSpinLimit = 1ll << 24;  // iterations before a device wait gives up (~1 s)

// Device-side status words.  err: 0 = ok, 1 = a grid barrier gave up
// (timeout), 2 = NaN/Inf met, 3 = Jacobi did not converge.
struct DevStatus {
  unsigned long long bar_count;  // grid-barrier arrivals (monotonic)
  unsigned long long bar_base;   // bar_count when the next cooperative kernel starts
  int err;
  int pad;
  unsigned int rot[3];  // Jacobi rotation counters, one per sweep modulo 3
  int pad2;             // sweeps taken by the last Jacobi launch
  unsigned long long pub_count;  // Householder reflectors published (monotonic)
  unsigned long long pub_base;   // pub_count when the next QR launch starts
  unsigned int pub_done;         // blocks of the current QR launch that have finished
  int pad3;
  long long wait_clocks;         // SM clocks a device-side wait spins before giving up (err = 1)
};

constexpr long long kDefaultWaitClocks = 2000000000ll;  // ~1 s at 2 GHz

// Grow-only device buffer owned by a context.
struct DevBuf {
  double* p = nullptr;
  size_t cap = 0;  // doubles
};

}  // namespace vp

struct vp_ctx {
  int device = 0;
  int num_sms = 0;
  int cluster_size = 0;  // CTAs per cluster for the cluster-resident kernels (16, or 8)
  int coop_cap = 0;      // max blocks of a cooperative grid launch (0: one per SM)
  int precision = 0;     // VP_PREC_* of the GEMM contractions (factorisations stay FP64)
  int modified_split = 0;  // > 0: compressions use the centre-bond-first scheme about this bond
  int grouped = 0;         // 1: the bond inside every (x_j, v_j) site pair is not truncated (IG ordering)
  long long wait_clocks = vp::kDefaultWaitClocks;  // limit of the device-side waits (DevStatus::wait_clocks)
  bool owns_stream = false;
  std::vector<vp_ctx*> children;  // contexts created for concurrent work
  cudaStream_t side = nullptr;     // side stream: Q formation beside the Jacobi SVD
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // QR sweep: site k factors into w_fac / w_p (k even) or w_fac_b / w_p_b (k
  // odd) and forms its Q on the side stream; ev_qf[b] = buffer b factored,
  // ev_qd[b] = its Q formed (buffer free again)
  vp::DevBuf w_fac_b, w_p_b;
  cudaEvent_t ev_qf[2] = {nullptr, nullptr}, ev_qd[2] = {nullptr, nullptr};
  cudaStream_t stream = nullptr;
  vp_alloc_fn alloc = nullptr;
  vp_free_fn freef = nullptr;
  cudaMemPool_t pool = nullptr;  // without caller allocator hooks: this context's pool (memory kept until destroy)
  void* user = nullptr;
  std::string err;
  int64_t launches = 0;
  vp::DevStatus* status = nullptr;  // device
  int* d_small = nullptr;           // device scratch ints (ranks, flags)
  int* h_small = nullptr;           // pinned host mirror
  double* d_smalld = nullptr;       // device scratch doubles
  double* h_smalld = nullptr;       // pinned host mirror
  // kernel-class timing
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  struct ProfMark {
    int cls;
    size_t ev;    // index of the begin event (the end event follows it)
    int m, n, k;  // shape of the launch (trace records)
  };
  std::vector<ProfMark> prof_marks;
  double prof_work[VP_K_COUNT] = {};
  int64_t prof_launches[VP_K_COUNT] = {};
  // workspaces
  vp::DevBuf w_fac, w_q, w_gemm, w_j, w_p, w_tmp, w_tmp2, w_vec, w_split;
  vp::DevBuf w_piv, w_q1, w_q2, w_r, w_p2, w_a, w_b, w_c, w_l;  // preconditioned SVD
  vp::DevBuf w_tca, w_tcb;            // packed operands of the tensor-core contractions
  vp::DevBuf w_q_side, w_split_side;  // scratch of the side-stream phase
  vp::DevBuf w_tca_side, w_tcb_side;
  std::vector<vp::DevBuf> w_chain;
  vp::DevBuf w_qrv;                   // double-word reflectors published by the grid QR kernel
  vp::DevBuf w_qrc;                   // its columns when they exceed shared memory
  vp::DevBuf w_fq, w_fq_side;         // double-word reflectors of the Q formation
  vp::DevBuf w_sig;                   // kept centre singular values (modified compression)
  vp::DevBuf w_wq, w_wr;              // wide QR: Q of the leading square block, R2^T
  // Blocks handed back to the caller's allocator only once the work queued
  // before their release has finished (the allocator callbacks know no
  // streams, and this context's kernels run on several).
  struct PendingFree {
    void* p;
    size_t bytes;
    cudaEvent_t ev;
  };
  std::vector<PendingFree> pending;
  std::vector<cudaEvent_t> free_events;
};

struct mps_t {
  vp_ctx* ctx = nullptr;
  int n = 0;
  std::vector<int> r;            // n+1 bonds
  std::vector<vp::DevBuf> core;  // core k: r[k]*2*r[k+1] doubles
};

struct mpo_t {
  vp_ctx* ctx = nullptr;
  int n = 0;
  std::vector<int> w;            // n+1 bonds
  std::vector<vp::DevBuf> core;  // core k: w[k]*4*w[k+1] doubles, (wl, out, in, wr)
};

namespace vp {

// ------------------------------------------------------------ host helpers
int fail(vp_ctx* ctx, int code, const std::string& msg);
int cuda_fail(vp_ctx* ctx, cudaError_t e, const char* what);
#define VP_CUDA(ctx, call)                                      \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return ::vp::cuda_fail(ctx, e_, #call); \
  } while (0)
#define VP_TRY(call)          \
  do {                        \
    int s_ = (call);          \
    if (s_ != VP_OK) return s_; \
  } while (0)

void* dev_alloc(vp_ctx* ctx, size_t bytes);
void dev_free(vp_ctx* ctx, void* p, size_t bytes);
// Make sure b holds at least `elems` doubles (contents not preserved).
int reserve(vp_ctx* ctx, DevBuf& b, size_t elems);
// Same, preserving the first `keep` doubles.
int reserve_keep(vp_ctx* ctx, DevBuf& b, size_t elems, size_t keep);
void release(vp_ctx* ctx, DevBuf& b);
// Return released blocks whose work has finished (all: wait for every one).
void drain_pending(vp_ctx* ctx, bool all);
int check_launch(vp_ctx* ctx, const char* what);
// Bracket one launch of class `cls` with events when profiling is on.
void prof_begin(vp_ctx* ctx, int cls);
void prof_end(vp_ctx* ctx, int cls, double work, int m = 0, int n = 0, int k = 0);
// Synchronise and read the device status word; maps errors to VP codes.
int sync_status(vp_ctx* ctx);
// Write ctx->wait_clocks into the device status words (stream-ordered).
int write_wait_limit(vp_ctx* ctx);

// Kernel attributes (dynamic shared memory limit, non-portable cluster size)
// set once per device for one kernel.  cudaFuncSetAttribute applies to the
// current device only, and the library's host threads (the second stream of
// a sim, species threads, batch workers) may launch the same kernel at once:
// a bit per device in an atomic mask, set under a mutex on first use.
struct AttrOnce {
  std::atomic<unsigned long long> done{0};
  int ensure(vp_ctx* ctx, const void* fn, int smem_bytes, bool cluster);
};

// ------------------------------------------------------------ kernels (linalg.cu)
// Row-major (m x n) -> column-major copy.
int launch_to_colmajor(vp_ctx* ctx, const double* A, int m, int n, double* out);
// In-place Householder QR of the column-major m x n matrix A (lda = m):
// R in the upper triangle, reflectors below, tau[min(m,n)].
int launch_qr_factor(vp_ctx* ctx, double* A, int m, int n, double* tau, double* vbuf);
// Kernel that factors an m x n matrix (shape and device only).
enum { QR_NONE = 0, QR_WIDE, QR_CDW, QR_CL, QR_GRID };
struct QRPlan {
  int kind;
  int cs;  // CTAs per cluster (QR_CDW, QR_CL)
};
QRPlan qr_plan(const vp_ctx* ctx, int m, int n);
// Q (m x p, p = min(m,n)) written row-major from the factored A.
int launch_qr_formq(vp_ctx* ctx, const double* A, int m, int n, const double* tau, double* Q);
// Upper-trapezoidal R (p x n) of the factored A, written row-major.
int launch_qr_getr(vp_ctx* ctx, const double* A, int m, int n, double* R);
// Output tile and split-K of a GEMM (shape and device only).
struct GemmPlan {
  int tile;    // 64 or 32
  int slices;  // K slices (1: no split)
  int kslice;  // columns of K per slice
};
GemmPlan gemm_plan(const vp_ctx* ctx, int M, int N, int K);
// C (M x N) = alpha * A (M x K) * B (K x N), all row-major with given leading dims.
int launch_gemm(vp_ctx* ctx, int M, int N, int K, double alpha, const double* A, int lda,
                const double* B, int ldb, double* C, int ldc);
// C (M x N) = A (M x K) * Bt^T, Bt given row-major (N x K).
int launch_gemm_bt(vp_ctx* ctx, int M, int N, int K, const double* A, int lda, const double* Bt, int ldbt,
                   double* C, int ldc);
// SVD preconditioning helpers (static pivoting by norm, see linalg.cu).
int launch_norm_order(vp_ctx* ctx, const double* M, int m, int c, int by_cols, int* piv);
int launch_gather_cm(vp_ctx* ctx, const double* M, int m, int c, const int* piv, int tall, double* out);
int launch_lower_from_upper(vp_ctx* ctx, const double* Rcm, int q, double* L);
int launch_scatter(vp_ctx* ctx, const double* Y, int rows, int cols_n, const int* piv, int cols, double* out);
int launch_svd_outputs_wide(vp_ctx* ctx, const double* X, const double* J, int b, int r, const int* perm,
                            double* Urows, double* Wv);
// Operand of a tensor-core contraction as (row, k) -> value: kind 0
// p[r * ld + k]; kind 1 p[k * ld + r]; kind 2 the upper triangle of a
// column-major factor, r <= k ? p[k * ld + r] : 0.
struct TcOperand {
  const double* p;
  int ld;
  int kind;
};
// C (M x N) = alpha * A (M x K) * B^T with B given as (N x K) operand, on the
// tensor cores in the context's reduced-precision mode (tcgemm.cu).
int launch_tc_gemm(vp_ctx* ctx, int M, int N, int K, double alpha, TcOperand a, TcOperand b, double* C, int ldc);
// C = alpha * triu(A_colmajor) (M x K) * B: the R factor read in place.
int launch_gemm_r(vp_ctx* ctx, int M, int N, int K, const double* Acm, int lda, const double* B,
                  int ldb, double* C, int ldc);
// One-sided Jacobi on the b rows (length c) of X, rotations also applied to
// the rows of J (b x b, set to the identity here).  Row-major, contiguous.
// floor_ok: the caller truncates every singular value below 1e-13 of the
// largest (tol >= 1e-13), so the double-word kernel, which leaves rows under
// 1e-15 of the largest unrotated, may be used.
int launch_jacobi_rows(vp_ctx* ctx, double* X, int b, int c, double* J, bool floor_ok);
// The same on a given stream with given status words.
int jacobi_rows_on(vp_ctx* ctx, cudaStream_t stream, DevStatus* status, double* X, int b, int c, double* J,
                   bool floor_ok);
// Largest cluster (16 or 8 CTAs, one per SM) the cluster-resident kernels
// can use on this device; 0 if none.
int probe_cluster_size();
// Sort row norms of X descending, choose the kept rank (chi, tol, ties),
// write perm/sigma/rank/truncation error into ctx scratch.  d_out[0] = rank.
int launch_select(vp_ctx* ctx, const double* X, int b, int c, int chi, double tol, int* perm,
                  double* sigma, int* d_rank, double* d_err);
// Vt (r x c) = X[perm[t]] / sigma[t];  W (b x r) = J[perm[t]][i] * sigma[t].
int launch_svd_outputs(vp_ctx* ctx, const double* X, const double* J, int b, int c, int r,
                       const int* perm, const double* sigma, double* Vt, double* W);

// ------------------------------------------------------------ kernels (mpsops.cu)
// out = alpha*a + beta*(B b) on one site (a may be NULL: pure apply; B may be
// NULL: identity).  See mps_axpby / mps_apply_mpo for the block layout.
struct SiteSum {
  const double* a; int al, ar;     // a core (al, 2, ar)
  const double* b; int bl, br;     // b core
  const double* B; int wl, wr;     // MPO core (wl, 2, 2, wr) or NULL
  double alpha, beta;
  int first, last;                 // site position flags
};
int launch_site_sum(vp_ctx* ctx, const SiteSum& s, double* out, int ol, int orr);
// T (rl x rr) = core[:,0,:] + core[:,1,:]
int launch_phys_sum(vp_ctx* ctx, const double* core, int rl, int rr, double* T);
int launch_copy(vp_ctx* ctx, const double* src, double* dst, size_t n);
// *out (device) = sum_i (a_i - b_i)^2 in a fixed order; scratch: 1024 doubles.
int launch_sqdiff(vp_ctx* ctx, const double* a, const double* b, size_t n, double* scratch, double* out);
// Status error 2 (VP_ENUMERIC at the next status read) if x holds a NaN or Inf.
int launch_check_finite(vp_ctx* ctx, const double* x, size_t n);
int launch_scale(vp_ctx* ctx, double* x, size_t n, double s);
// Core (a, 2, b) -> (b, 2, a): the site read in the opposite chain direction.
int launch_core_transpose(vp_ctx* ctx, const double* in, int a, int b, double* out);
// Rows of a row-major (rows x cols) matrix scaled by sv (or 1/sv, 0 for 0).
int launch_scale_rows(vp_ctx* ctx, double* x, int rows, int cols, const double* sv, int invert);
// dense f[ix][iv] -> site-ordered vector (gather) and back.
int launch_permute_to_sites(vp_ctx* ctx, const double* f, int nx, int nv, int mapping, double* out,
                            int inverse);
int launch_poisson(vp_ctx* ctx, const double* rho, int N, double dx, double* E, double* we_dev);
// Several species: net density sum_s w[s] rho[s][i] and masses sum rho_s dx.
constexpr int kMaxSpecies = 16;
struct SpeciesRho {
  const double* rho[kMaxSpecies];
  double w[kMaxSpecies];
  int ns;
};
int launch_species_net(vp_ctx* ctx, const SpeciesRho& sr, int N, double dx, double* net, double* mass);
// MPO core on one site for the E-term diag(E) (x) D_v (placed product).
struct ETermSite {
  int is_x;                 // site carries an x bit
  const double* Ecore;      // x site: E core (el, 2, er)
  int el, er;
  const double* Dcore;      // v site: D_v core (dl, 2, 2, dr)
  int dl, dr;
  int ew, dw;               // bond of the other dimension carried through
};
// Fill L core = blockdiag(U core, E-term core) (first/last concatenation).
int launch_assemble_site(vp_ctx* ctx, const double* U, int ul, int ur, const ETermSite& e, int first,
                         int last, double* out, int ol, int orr);
// ------------------------------------------------------------ batched launches
// One launch serves up to kMaxBatch independent problems of one kind: the
// same sweep position of several compressions, or the same step of several
// simulations.  The per-problem arguments travel in the kernel's parameter
// block (Pack), the problem index is a grid coordinate, and every problem
// runs the kernel variant and launch geometry its own single launch would
// use, so its arithmetic does not depend on the batch.  Launchers take the
// problems as a vector, split it into packs and, where the single path picks
// a kernel variant by shape, into one launch per variant; problems that no
// batched kernel serves (factors beyond a cluster's shared memory) run one
// by one.  Per-problem scratch comes from a BScratch owned by the caller.
constexpr int kMaxBatch = 32;
template <class A>
struct Pack {
  A a[kMaxBatch];
};

// Several jobs of one launcher call may name the same BScratch (the two Q
// formations of an SVD site, its output GEMMs): each takes its own slot.
constexpr int kScratchSlots = 4;
struct BScratch {
  DevBuf wq, wr;                  // wide QR: Q of the square block, R2^T
  DevBuf qrv, qrc;                // grid QR: published reflectors, columns beyond shared memory
  DevBuf fq[kScratchSlots];       // Q formation: double-word reflectors
  DevBuf qscr[kScratchSlots];     // Q formation: column scratch (m > 512)
  DevBuf split[kScratchSlots];    // GEMM split-K partial products
  DevStatus* st = nullptr;        // status words of the problem (device)
};
void release_scratch(vp_ctx* ctx, BScratch& s);

struct BColMajor { const double* A; int m, n; double* out; };
struct BQR { double* A; int m, n; double* tau; double* vbuf; BScratch* s; };
struct BFormQ { const double* A; int m, n; const double* tau; double* Q; BScratch* s; };
struct BGetR { const double* A; int m, n; double* R; };
enum { BG_AB = 0, BG_ABT = 1, BG_RB = 2 };  // A row-major x B row-major / B^T given / triu(A col-major) x B
struct BGemm {
  int kind;  // BG_*
  int fp32;  // FP32 contraction mode
  int M, N, K;
  double alpha;
  const double* A; int lda;
  const double* B; int ldb;
  double* C; int ldc;
  BScratch* s;
};
struct BNormOrder { const double* M; int m, c, by_cols; int* piv; };
struct BGather { const double* M; int m, c; const int* piv; int tall; double* out; };
struct BLowerUpper { const double* R; int q; double* L; };
struct BCopy { const double* src; double* dst; size_t n; };
struct BJacobi { double* X; int b, c; double* J; DevStatus* st; };
struct BSelect {
  const double* X; int b, c, chi; double tol; int* perm; double* sigma; int* d_rank; double* d_err; DevStatus* st;
};
struct BSvdOut { const double* X; const double* J; int b, c, r; const int* perm; const double* sigma; double* Vt; double* W; };
struct BSvdOutWide { const double* X; const double* J; int b, r; const int* perm; double* U; double* Wv; };
struct BScatter { const double* Y; int rows, cols_n; const int* piv; int cols; double* out; };

int blaunch_to_colmajor(vp_ctx* ctx, cudaStream_t st, const std::vector<BColMajor>& v);
int blaunch_qr_factor(vp_ctx* ctx, cudaStream_t st, const std::vector<BQR>& v);
int blaunch_qr_formq(vp_ctx* ctx, cudaStream_t st, const std::vector<BFormQ>& v);
int blaunch_qr_getr(vp_ctx* ctx, cudaStream_t st, const std::vector<BGetR>& v);
int blaunch_gemm(vp_ctx* ctx, cudaStream_t st, const std::vector<BGemm>& v);
int blaunch_norm_order(vp_ctx* ctx, cudaStream_t st, const std::vector<BNormOrder>& v);
int blaunch_gather_cm(vp_ctx* ctx, cudaStream_t st, const std::vector<BGather>& v);
int blaunch_lower_from_upper(vp_ctx* ctx, cudaStream_t st, const std::vector<BLowerUpper>& v);
// Jacobi of truncating compressions (tol >= 1e-13: the double-word kernel).
int blaunch_jacobi(vp_ctx* ctx, cudaStream_t st, const std::vector<BJacobi>& v);
int blaunch_select(vp_ctx* ctx, cudaStream_t st, const std::vector<BSelect>& v);
int blaunch_svd_outputs(vp_ctx* ctx, cudaStream_t st, const std::vector<BSvdOut>& v);
int blaunch_svd_outputs_wide(vp_ctx* ctx, cudaStream_t st, const std::vector<BSvdOutWide>& v);
int blaunch_scatter(vp_ctx* ctx, cudaStream_t st, const std::vector<BScatter>& v);

// mpsops.cu
struct BSiteSum { SiteSum s; double* out; int ol, orr; };
struct BPhysSum { const double* core; int rl, rr; double* T; };
struct BScale { double* x; size_t n; double s; };
struct BPoisson { const double* rho; int N; double dx; double* E; double* we; };
struct BAssemble { const double* U; int ul, ur; ETermSite e; int first, last; double* out; int ol, orr; };
struct BPermute { const double* f; int nx, nv, mapping; double* out; int inverse; };
struct BCheck { const double* x; size_t n; DevStatus* st; };
int blaunch_check_finite(vp_ctx* ctx, cudaStream_t st, const std::vector<BCheck>& v);
int blaunch_copy(vp_ctx* ctx, cudaStream_t st, const std::vector<BCopy>& v);
int blaunch_site_sum(vp_ctx* ctx, cudaStream_t st, const std::vector<BSiteSum>& v);
int blaunch_phys_sum(vp_ctx* ctx, cudaStream_t st, const std::vector<BPhysSum>& v);
int blaunch_scale(vp_ctx* ctx, cudaStream_t st, const std::vector<BScale>& v);
int blaunch_poisson(vp_ctx* ctx, cudaStream_t st, const std::vector<BPoisson>& v);
int blaunch_assemble(vp_ctx* ctx, cudaStream_t st, const std::vector<BAssemble>& v);
int blaunch_permute(vp_ctx* ctx, cudaStream_t st, const std::vector<BPermute>& v);

// MPO -> dense (small n), and MPS eval helpers
int launch_mpo_dense_step(vp_ctx* ctx, const double* T, int rows, int cols, int w, const double* core,
                          int wr, double* out);

}  // namespace vp
