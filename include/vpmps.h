/*
 * vpmps.h -- C ABI of the GB300 matrix-product-state Vlasov-Poisson library.
 *
 * Method: Ye & Loureiro, "A quantum-inspired method for solving the
 * Vlasov-Poisson equations" (arXiv:2205.11990).  A 1D1V distribution f(x,v)
 * on a 2^nx x 2^nv grid is stored as a quantized tensor train (MPS, one bit
 * per site, Sec. "MPS Representation of Classical Data"); one time step
 * applies the finite-difference MPOs (SI "Derivatives", "Upwind time
 * evolution"), adds MPS (SI "Addition"), integrates over v (SI
 * "Integration"), solves Poisson for E (Eq. 2-3 of "Problem Statement") and
 * recompresses with a QR canonicalisation sweep followed by a truncated SVD
 * sweep (SI "Canonicalization and Compression"), inside RK4 with compression
 * level C1 (SI "Compressed time evolution algorithm").
 *
 * Conventions
 *  - Every function returns an int status (VP_OK = 0); vp_last_error() gives
 *    a one-line description of the last failure on a context.
 *  - Precision.  Every array in memory (MPS and MPO cores, densities,
 *    fields) is IEEE FP64, and so are the contractions (MPO x MPS, the GEMMs
 *    of the sweeps in the default VP_PREC_FP64 mode), the Poisson solve and
 *    the truncation rule.  The latency-bound factorisations of the
 *    compression sweeps -- Householder QR, the formation of Q and the
 *    truncating one-sided Jacobi SVD -- compute in double-word FP32
 *    arithmetic (each value the unevaluated sum of two floats, about 48
 *    significant bits, unit roundoff ~2^-48 instead of FP64's 2^-53) behind
 *    exact power-of-two prescaling; they read and write FP64.  Against an
 *    FP64 LAPACK implementation of the same method this leaves f within
 *    ~1e-12 relative (L2) and the field energy within ~1e-12 relative per
 *    step.  Compressions with tol = 0 (exact mode) use an FP64 Jacobi SVD.
 *    No function falls back to the CPU: without a usable CUDA device
 *    vp_ctx_create fails with VP_ECUDA.
 *  - Handles (vp_ctx, mps_t, mpo_t, vp_sim) are opaque and owned by the
 *    caller: each *_create has a matching *_destroy.  MPS/MPO/sim objects
 *    must be destroyed before their context.
 *  - Device memory is the library's, obtained through the allocator passed to
 *    vp_ctx_create (or cudaMallocAsync on the context's stream when NULL).
 *    Pointers documented as "host" are caller-owned host buffers; "device"
 *    pointers are caller-owned device buffers on the context's device.
 *  - Work is enqueued on the context's CUDA stream.  Functions that return
 *    host data synchronise that stream before returning.  A context is not
 *    re-entrant: use one context per host thread / stream.
 *  - Site ordering (main text, "State Compressibility"): x_0 / v_0 is the most
 *    significant (coarsest) bit of a dimension.  VP_SEQ (S1): x_0..x_{nx-1},
 *    v_0..v_{nv-1}; VP_SEQ_S2: x_{nx-1}..x_0 (fine to coarse), then
 *    v_0..v_{nv-1}; VP_SEQ_S3: x_0..x_{nx-1}, then v_{nv-1}..v_0;
 *    VP_INTERLEAVED (IF): x_0, v_0, x_1, v_1, ..., leftover bits of the longer
 *    dimension last.  VP_INTERLEAVED_GROUPED (IG, nx == nv): the grouped
 *    interleaved ordering, each (x_j, v_j) pair one site of dimension 4.  It
 *    is held in the IF site order with the bond inside every pair left
 *    untruncated (kept to 1e-13, never capped at chi): the same state and the
 *    same truncations at the pair bonds as d = 4 cores.  Bond lists and
 *    entropies then have the pair bonds at the even positions of the IF
 *    list (after sites 1, 3, 5, ...).  The IG rule applies to mps_create and
 *    to every compression of a sim or multi-species run on an IG layout.
 *  - Grid: x_i = xmin + i dx, dx = (xmax - xmin)/2^nx (periodic, right end
 *    excluded); v_j = vmin + j dv, dv = (vmax - vmin)/(2^nv - 1) (both ends
 *    included, zero-gradient boundaries).  The v domain must be symmetric
 *    (vmin = -vmax) so that v > 0 exactly on the upper half of the v grid.
 *  - Dense arrays f are row-major f[ix * 2^nv + iv] (double).
 */
#ifndef VPMPS_H
#define VPMPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  VP_OK = 0,
  VP_EINVAL = 1,     /* bad argument (sizes, NULL, unsupported layout) */
  VP_ENOMEM = 2,     /* allocator returned NULL */
  VP_ECAPACITY = 3,  /* a bond or workspace exceeds a documented limit */
  VP_ECUDA = 4,      /* CUDA runtime error (message in vp_last_error) */
  VP_ETIMEOUT = 5,   /* a device-side wait gave up after its iteration limit */
  VP_ENUMERIC = 6,   /* NaN/Inf in singular values or the field */
  VP_ECFL = 7,       /* time step above the RK4 stability limit */
  VP_EBUSY = 8,      /* object in use by another operation */
  VP_EIO = 9         /* checkpoint file missing, unreadable or malformed */
};

enum { VP_SEQ = 0, VP_INTERLEAVED = 1, VP_SEQ_S2 = 2, VP_SEQ_S3 = 3, VP_INTERLEAVED_GROUPED = 4 };

/* Opaque handles. */
typedef struct vp_ctx vp_ctx;
typedef struct mps_t mps_t;
typedef struct mpo_t mpo_t;
typedef struct vp_sim vp_sim;

/* Device allocator hooks: alloc returns device memory of at least `bytes`
 * bytes usable on the context's stream (NULL on failure); free releases it. */
typedef void* (*vp_alloc_fn)(size_t bytes, void* user);
typedef void (*vp_free_fn)(void* ptr, size_t bytes, void* user);

typedef struct {
  int nx, nv;      /* bits per dimension, each in [2, 14] */
  int mapping;     /* VP_SEQ, VP_INTERLEAVED, VP_SEQ_S2, VP_SEQ_S3 or VP_INTERLEAVED_GROUPED */
  double xmin, xmax, vmin, vmax;
} vp_layout;

/* ---------------------------------------------------------------- context */

/* Create a context on the current CUDA device.  `cuda_stream` is a
 * cudaStream_t (NULL = legacy default stream).  alloc/free may both be NULL
 * (stream-ordered cudaMallocAsync/cudaFreeAsync).  Errors: VP_EINVAL,
 * VP_ECUDA (no device). */
int vp_ctx_create(void* cuda_stream, vp_alloc_fn alloc, vp_free_fn free_fn, void* user,
                  vp_ctx** out);
int vp_ctx_destroy(vp_ctx* ctx);
const char* vp_last_error(const vp_ctx* ctx);
/* Arithmetic-rate probes (no counterpart in the paper; diagnostics for the
 * roofline of the kernels): the measured throughput, TFLOP/s of FP64-
 * equivalent flops, of one unit kind on this device -- VP_PROBE_FP64_FMA
 * (FP64 FMA, 2 flops), VP_PROBE_FP32_FMA (FP32 FMA, 2 flops),
 * VP_PROBE_DW_DOT (one double-word compensated dot-product step, 12 FP32
 * instructions, 2 flops), VP_PROBE_DW_AXPY (one double-word c - w v element,
 * 29 FP32 instructions, 2 flops), VP_PROBE_DMMA (FP64 mma.sync m8n8k4).  One
 * warm-up and one timed launch of ~10 ms on the context's stream; no device
 * setting is touched.  Errors: VP_EINVAL, VP_ENOMEM, VP_ECUDA. */
enum { VP_PROBE_FP64_FMA = 0, VP_PROBE_FP32_FMA = 1, VP_PROBE_DW_DOT = 2, VP_PROBE_DW_AXPY = 3, VP_PROBE_DMMA = 4 };
int vp_peak_probe(vp_ctx* ctx, int kind, double* tflops_out);

/* Failure detection (no counterpart in the paper).  The device-side waits of
 * the cooperative kernels (the grid barrier, the published-reflector counter
 * of the grid QR) spin at most `clocks` SM clocks (default 2e9, ~1 s; 0
 * restores it) before they give up: the kernel records the timeout and
 * returns, and the call that launched it fails with VP_ETIMEOUT while the
 * context stays usable (its status words are reset).  A small limit is a
 * way to exercise that path without a real fault; it also applies to the
 * contexts this one creates for concurrent work.  Synchronises the stream.
 * Errors: VP_EINVAL (clocks < 0). */
int vp_ctx_set_wait_limit(vp_ctx* ctx, long long clocks);
/* Number of kernels this context has launched so far (diagnostics). */
int64_t vp_kernel_launches(const vp_ctx* ctx);

/* Kernel-class timing (diagnostics): while enabled, every launch of the
 * classes below is bracketed by CUDA events on the context's stream.
 * vp_profile_enable clears the counters; vp_profile_read synchronises and
 * returns the summed event time (ms), the launch count and the algorithmic
 * work of the class (FP64 flops for VP_K_QR..VP_K_JACOBI, bytes moved for
 * VP_K_APPLY). */
enum { VP_K_QR = 0, VP_K_FORMQ = 1, VP_K_GEMM = 2, VP_K_JACOBI = 3, VP_K_SELECT = 4, VP_K_APPLY = 5,
       VP_K_OTHER = 6, VP_K_COUNT = 7 };
int vp_profile_enable(vp_ctx* ctx, int on);
int vp_profile_read(vp_ctx* ctx, int kclass, double* ms, int64_t* launches, double* work);
/* Launch trace of the same profiling window: one record per bracketed
 * launch, in issue order (this context first, then the contexts it created
 * for concurrent work).  m, n, k: the shape of the launch (QR: rows, columns;
 * Jacobi: rows, row length, sweeps taken; GEMM: M, N, K; apply: the site).
 * With concurrent streams an event interval also counts time spent queued
 * behind the other stream's kernels; with one stream it is the kernel's own
 * time.  Writes up to `cap` records, *n_out = the total available. */
typedef struct {
  int kclass;
  int m, n, k;
  double ms;
} vp_trace_rec;
int vp_profile_trace(vp_ctx* ctx, vp_trace_rec* out, int cap, int* n_out);

/* -------------------------------------------------------------------- MPS */

/* a1: f (2^(nx+nv) doubles, row-major f[ix][iv]; host if f_on_device == 0,
 * else device) -> MPS.  Exact left-canonical decomposition by a chain of
 * Householder QR factorisations (iterated decomposition of reshapes, Sec.
 * "MPS Representation", Fig. 1a), then the truncated-SVD sweep with bond cap
 * chi and tolerance tol (truncation-error equation, Sec. "MPS
 * Representation").  Errors: VP_EINVAL (layout), VP_ENOMEM, VP_ENUMERIC (a
 * NaN or Inf in f). */
int mps_create(vp_ctx* ctx, const vp_layout* layout, const double* f, int f_on_device, int chi,
               double tol, mps_t** out);

/* MPS from raw cores (host).  ranks[0..n] with ranks[0] = ranks[n] = 1; the
 * cores are packed site after site, core k row-major (ranks[k], 2,
 * ranks[k+1]).  No truncation. */
int mps_create_cores(vp_ctx* ctx, int n, const int* ranks, const double* cores_host, mps_t** out);
int mps_destroy(mps_t* mps);
int mps_num_sites(const mps_t* mps);
/* ranks_out: n+1 ints (host). */
int mps_bonds(const mps_t* mps, int* ranks_out);
/* Packed cores to host (layout as mps_create_cores); `capacity` doubles. */
int mps_get_cores(vp_ctx* ctx, const mps_t* mps, double* host_out, size_t capacity);
/* Checkpoint an MPS to a file / restore it (the state is the whole of a
 * simulation's f, so a run can resume from it).  File: 8-byte magic
 * "VPMPS01\0", int32 n, int32 0, int32 ranks[n+1], zero padding to 8 bytes,
 * then the cores packed as in mps_get_cores (FP64), little-endian.  mps_save
 * writes `path`.tmp and renames it over `path`; mps_load rejects a file whose
 * size disagrees with its bond ranks before it allocates anything.  Errors: VP_EIO (open/read/write or
 * format), VP_EINVAL, VP_ENOMEM. */
int mps_save(vp_ctx* ctx, const mps_t* mps, const char* path);
int mps_load(vp_ctx* ctx, const char* path, mps_t** out);
/* Validate a checkpoint file without loading it (host only, no context, no
 * GPU): magic, header, bond ranks (1 <= r <= 2^20, boundary ranks 1) and a
 * file size equal to header + 8 * payload elements; the header is checked
 * before anything is allocated.  n_out (may be NULL): number of sites;
 * ranks_out (may be NULL): n+1 ints (at most 65); elems_out (may be NULL):
 * FP64 payload elements.  Errors: VP_EINVAL (NULL path), VP_EIO. */
int mps_file_info(const char* path, int* n_out, int* ranks_out, size_t* elems_out);
/* Contract to the dense 2^n vector indexed by site bits (site 0 = MSB), host
 * output.  n <= 24. */
int mps_to_dense(vp_ctx* ctx, const mps_t* mps, double* host_out);
/* Same as a dense f[ix][iv] array for the given layout (undoes the site
 * permutation of VP_INTERLEAVED). */
int mps_to_grid(vp_ctx* ctx, const mps_t* mps, const vp_layout* layout, double* host_out);

/* -------------------------------------------------------------------- MPO */

enum {
  VP_MPO_DX_CENTERED = 0,   /* SI "First Derivative, Centered, Periodic" on the x bits */
  VP_MPO_DX_FORWARD = 1,    /* SI "First Derivative, Forward, Periodic" */
  VP_MPO_DX_BACKWARD = 2,   /* SI "First Derivative, Backward, Periodic" */
  VP_MPO_DV_ZERO_GRAD = 3,  /* SI "First Derivative, Centered, Zero Gradient" on the v bits */
  VP_MPO_DXX = 4,           /* SI "Second Derivative, Centered, Periodic" on the x bits */
  VP_MPO_ADVECTION = 5      /* -v+ D_b^x - v- D_f^x (SI "Upwind time evolution") */
};

/* Build one of the operators above on the full site chain of `layout`
 * (identity on the other dimension).  Errors: VP_EINVAL. */
int mpo_create_vp(vp_ctx* ctx, const vp_layout* layout, int kind, mpo_t** out);
/* L(E) = -v+ D_b^x - v- D_f^x + diag(E) D_c^v with E (2^nx doubles, host) as
 * an MPS truncated at e_tol (no bond cap). */
int mpo_create_vlasov(vp_ctx* ctx, const vp_layout* layout, const double* E_host, double e_tol,
                      mpo_t** out);
/* MPO from raw cores (host): bonds[0..n], core k row-major (bonds[k], 2_out,
 * 2_in, bonds[k+1]). */
int mpo_create_cores(vp_ctx* ctx, int n, const int* bonds, const double* cores_host, mpo_t** out);
int mpo_destroy(mpo_t* mpo);
int mpo_num_sites(const mpo_t* mpo);
/* bonds_out: n+1 ints (host). */
int mpo_bonds(const mpo_t* mpo, int* bonds_out);
/* Dense 2^n x 2^n operator [out][in] (site-bit indices), host; n <= 12. */
int mpo_to_dense(vp_ctx* ctx, const mpo_t* mpo, double* host_out);

/* ------------------------------------------------------------ operations */

/* a6: out = mpo * in, per-site contraction C(o) = sum_i B(o,i) A(i), bond
 * gamma = (alpha, beta) (SI "Matrix-vector multiplication").  No
 * truncation; out bonds = in bonds * mpo bonds.  `out` is overwritten. */
int mps_apply_mpo(vp_ctx* ctx, const mpo_t* mpo, const mps_t* in, mps_t* out);

/* a7: out = a*x + b*y with block-diagonal cores (SI "Addition"). */
int mps_axpby(vp_ctx* ctx, double a, const mps_t* x, double b, const mps_t* y, mps_t* out);

/* a8+a9: QR sweep left to right (R into the next core), then truncated-SVD
 * sweep right to left keeping r = min(chi, r_tol) singular values per bond,
 * r_tol the smallest r whose normalised tail sqrt(sum_{i>r} s_i^2)/||s|| is
 * <= tol (tol = 0: no tolerance cut); a cut that would split a cluster of
 * values within a relative 1e-5 of each other moves to the cluster start.
 * trunc_err_out: n-1 doubles (host) or NULL.  Errors: VP_ETIMEOUT,
 * VP_ENUMERIC. */
int mps_compress(vp_ctx* ctx, mps_t* inout, int chi, double tol, double* trunc_err_out);
/* Compressibility diagnostic (main text, "State Compressibility", the rms
 * compression error against the bond dimension D): for each chi[i] a copy of
 * f compressed with bond cap chi[i] and tolerance tol (mps_compress), and
 * rms_out[i] = sqrt(sum_j (f_j - f_D,j)^2 / 2^n), the rms difference of the
 * two dense vectors over all 2^n grid points, summed on the GPU in a fixed
 * order (never from MPS overlaps, which cancel catastrophically).  f is not
 * changed.  n <= 24.  rms_out: nchi doubles (host).  Errors: VP_EINVAL. */
int mps_compression_error(vp_ctx* ctx, const mps_t* f, int nchi, const int* chi, double tol, double* rms_out);
/* Modified centre-bond-first compression (SI "Modified Compression Scheme")
 * about the bond after site split-1 (1 <= split < n; for a sequential
 * ordering, split = nx is the x / v cut): the bond is put at the centre of a
 * mixed canonical form and truncated first (chi, tol as for mps_compress),
 * S^{-1} S is inserted there, the two halves are swept outward from it with
 * the same truncation rule, and S^{-1} is absorbed into site split.  The
 * result is not in canonical form.  trunc_err_out as for mps_compress.
 * Errors: VP_EINVAL. */
int mps_compress_modified(vp_ctx* ctx, mps_t* inout, int split, int chi, double tol, double* trunc_err_out);

/* a3: rho[ix] = sum_iv f(x_ix, v_iv) dv (SI "Integration", rectangle rule);
 * rho_dev: 2^nx doubles (device). */
int vp_density(vp_ctx* ctx, const vp_layout* layout, const mps_t* f, double* rho_dev);

/* a4: periodic second-order Poisson d2phi/dx2 = rho - mean(rho) (zero-mean
 * phi), E = -(phi_{i+1} - phi_{i-1})/(2 dx).  rho_dev, E_dev: 2^nx doubles
 * (device); field_energy_host: 1/2 sum E^2 dx (host) or NULL. */
int vp_poisson(vp_ctx* ctx, const double* rho_dev, int nx, double dx, double* E_dev,
               double* field_energy_host);

/* Allocation-free variant of vp_poisson (no counterpart in the paper; a
 * deployment aid).  For callers that cannot allocate device memory and so
 * cannot create a vp_ctx -- code running under another framework's fixed
 * memory budget, or a thread that must not touch the allocator while a graph
 * capture is in progress elsewhere.  Inputs and outputs are the caller's:
 * rho_dev, E_dev (2^nx doubles, device), field_energy_host / mass_host (host,
 * may be NULL).  Its scratch is a file-scope device array of 16384 + 64
 * doubles (~128 KB) that every GPU which loads the library keeps until the
 * process exits; nothing in it needs clearing between calls (each call writes
 * every element it reads).  All calls on a device share that array, so calls
 * that overlap on the GPU race: serialise them (one stream, or events).  The
 * first call on a device is its set-up: it looks up the array's device
 * address (cudaGetSymbolAddress with that device current), and under CUDA's
 * lazy module loading that lookup can load the library's device code, which
 * may itself allocate device memory for the module.  So make one call (any
 * valid size) during the caller's own set-up, before its no-allocation phase
 * and before any stream capture; every later call on that device allocates
 * nothing.  `cuda_stream` must belong to the current device (VP_EINVAL
 * otherwise).  Errors: VP_EINVAL, VP_ECAPACITY (nx > 14: 2^nx beyond the
 * static scratch), VP_ECUDA.  Synchronises `cuda_stream` when a host output
 * is requested. */
int vp_poisson_noalloc(void* cuda_stream, const double* rho_dev, int nx, double dx, double* E_dev,
                       double* field_energy_host, double* mass_host);

/* Dense contraction C (M x N) = alpha * A (M x K) * B (K x N), row-major
 * device buffers with leading dimensions lda >= K, ldb >= N, ldc >= N, in
 * the arithmetic of `precision` (VP_PREC_*, see vp_config): the kernel the
 * sweeps use for their GEMM-shaped contractions (R x next core, U S
 * products).  K = 0 gives C = 0.  Synchronises the context stream; a device
 * wait that gave up is reported as VP_ETIMEOUT.  Errors: VP_EINVAL. */
int vp_gemm(vp_ctx* ctx, int precision, int M, int N, int K, double alpha, const double* A, int lda,
            const double* B, int ldb, double* C, int ldc);

/* --------------------------------------------------------------- stepping */

typedef struct {
  double dt;        /* fixed step; must satisfy vmax*dt/dx <= 0.6963 (else VP_ECFL) */
  int chi;          /* bond cap of f_{n+1} */
  double tol;       /* truncation tolerance of every compression (1e-10) */
  double e_tol;     /* tolerance of the E-field MPS (1e-10) */
  int streams;      /* 1: one stream; 2: the two independent compressions of
                       each RK stage run concurrently on a second stream;
                       0: the step runs as a one-member lockstep group
                       (vp_group_*: both compressions of a stage share every
                       launch) where the configuration allows it (level C1,
                       plain sweeps, FP64 or FP32 contractions, tol and e_tol
                       >= 1e-13), else as 2.  The result is the same in
                       every mode. */
  int level;        /* compression level (SI "Compressed time evolution
                       algorithm"), 0 or 1: C1; 2..5: C2..C5 -- C2 also caps the
                       intermediate states at chi, C3 also the running sum of
                       derivatives (D = k1, D <- C(D + w_i k_i), w = 2, 2, 1;
                       f_{n+1} = C(f_n + dt/6 D)), C4 also each derivative,
                       C5 also the advection and field terms of each
                       derivative before they are added */
  int e_chi;        /* bond cap D_F of the field MPS (main text, "Approximation
                       of the nonlinear term"); 0: no cap */
  int precision;    /* VP_PREC_*: arithmetic of the dense contractions of the
                       sweeps (R x next core, the Q and U S products).  The
                       other steps do not change with the mode: the MPO
                       application, the truncation rule and the Poisson
                       solve stay FP64, and the QR, Q formation and Jacobi
                       SVD stay in double-word FP32 (~2^-48, see the
                       precision convention at the top of this file).
                         FP64          FP64 FMA;
                         FP32_CONTRACT FP32 FMA, FP32 accumulation (CUDA cores);
                         TF32          tensor cores, operands rounded to TF32,
                                       FP32 accumulation in tensor memory;
                         BF16          tensor cores, BF16 operands, FP32
                                       accumulation;
                         TF32X3        tensor cores, split products
                                       a_hi b_hi + a_hi b_lo + a_lo b_hi of
                                       TF32 halves, FP32 accumulation. */
  int compression;  /* VP_COMPRESS_SWEEPS (0): QR sweep then truncated-SVD
                       sweep (SI "Canonicalization and Compression");
                       VP_COMPRESS_MODIFIED (1): the centre-bond-first scheme
                       of SI "Modified Compression Scheme" for every
                       compression of the step, centred on the x / v bond
                       (sequential orderings only, else VP_EINVAL) */
} vp_config;

enum { VP_COMPRESS_SWEEPS = 0, VP_COMPRESS_MODIFIED = 1 };

enum {
  VP_PREC_FP64 = 0,
  VP_PREC_FP32_CONTRACT = 1,
  VP_PREC_TF32 = 2,
  VP_PREC_BF16 = 3,
  VP_PREC_TF32X3 = 4
};

typedef struct {
  double t;             /* time at the start of the step */
  double field_energy;  /* W_E = 1/2 sum E^2 dx of f_n */
  double mass;          /* sum f dx dv of f_n */
  int max_bond;         /* max bond of f_{n+1} */
  double trunc_err;     /* max per-bond truncation error of the final compression */
} vp_record;

/* a10: RK4 stepper with compression level C1.  The sim copies f0. */
int vp_sim_create(vp_ctx* ctx, const vp_layout* layout, const vp_config* cfg, const mps_t* f0,
                  vp_sim** out);
int vp_sim_destroy(vp_sim* sim);
/* Advance nsteps; records[nsteps] (host) receives a11 diagnostics or NULL. */
int vp_step(vp_sim* sim, int nsteps, vp_record* records);
/* The current state (owned by the sim; valid until the next vp_step). */
const mps_t* vp_sim_state(const vp_sim* sim);
/* Entanglement entropy per bond (main text, EE equation: -sum p log2 p over
 * the normalised squared singular values kept at that bond) of the last step's
 * final compression; S_out: n-1 doubles (host).  Zero before the first step. */
int vp_sim_entropy(const vp_sim* sim, double* S_out);
/* Algorithmic FP64 flop count of the factorisations since creation. */
double vp_sim_flops(const vp_sim* sim);

/* f0 (host dense) -> nsteps of RK4-C1 -> f(T) dense (host, may be NULL) and
 * records[nsteps] (host, may be NULL). */
int vp_run(vp_ctx* ctx, const vp_layout* layout, const vp_config* cfg, const double* f0_host,
           int nsteps, double* fT_host, vp_record* records);

/* -------------------------------------------- lockstep groups of sims */

/* One RK4-C1 step of many independent simulations at once (no counterpart in
 * the paper: the batching layer around its time stepper).  Every kernel
 * launch of a group step serves all members at the same position of the
 * step -- the MPO x MPS contractions and sums of every site (SI
 * "Matrix-vector multiplication", "Addition"), the Householder QR and the
 * preconditioned Jacobi SVD of the same sweep site of every member's
 * compressions (SI "Canonicalization and Compression"), the densities,
 * Poisson solves and field MPS (SI "Integration", "Dot Product") -- and the
 * host waits once per SVD site for the kept ranks of all members instead of
 * once per member.  Members may differ in grid bits, mapping, chi, tol and
 * dt; members with fewer sites simply sit out the sweep positions they do not
 * have.  Each member runs the kernel variants and launch geometries of its
 * own vp_step, so its result does not depend on the group.
 *
 * Members are sims created with vp_sim_create on the group's context with
 * cfg.streams = 1, compression level C1 (cfg.level 0 or 1), the plain sweeps
 * (VP_COMPRESS_SWEEPS), precision VP_PREC_FP64 or VP_PREC_FP32_CONTRACT and
 * tol, e_tol >= 1e-13.  A group holds no reference to a member's memory
 * beyond its workspaces: remove a sim before destroying it. */
typedef struct vp_group vp_group;
/* Errors: VP_EINVAL (max_members outside 1..4096), VP_ENOMEM, VP_ECUDA. */
int vp_group_create(vp_ctx* ctx, int max_members, vp_group** out);
/* Append a member (member index = number of members before the call).
 * Errors: VP_EINVAL (sim not eligible, see above, or already a member),
 * VP_ECAPACITY (group full). */
int vp_group_add(vp_group* g, vp_sim* sim);
/* Remove a member; the members after it move down one index. */
int vp_group_remove(vp_group* g, vp_sim* sim);
int vp_group_size(const vp_group* g);
/* Advance every running member by one step.  records[i] (host, size() or
 * NULL) receives member i's a11 diagnostics as vp_step would; status[i]
 * (host, size() or NULL) its state: VP_OK, or the error that stopped it --
 * VP_ENUMERIC (NaN/Inf or a Jacobi that did not converge in its own
 * arithmetic) or VP_ETIMEOUT (a device wait of its own gave up).  A member
 * that failed stops there, the others go on, and it stays stopped (its state
 * undefined) until removed.  The return value is VP_OK unless the group's
 * own launches failed (VP_ENOMEM, VP_ECUDA, ...), which stops every member.
 * Synchronises the context's stream. */
int vp_group_step(vp_group* g, vp_record* records, int* status);
/* Batched a1: `count` MPS at once (count <= 2 max_members), each exactly as
 * mps_create would make it from the host grid f_host[i] on layouts[i] (site
 * permutation, decomposition by a chain of Householder QR factorisations,
 * truncated-SVD sweep with chi[i], tol[i]; the IG pair rule on IG layouts),
 * with every factorisation of the same site of all grids in one batched
 * launch.  out[i] receives the new MPS (owned by the caller, on the group's
 * context) or NULL; status[i] VP_OK or the error of grid i alone (VP_EINVAL:
 * bad layout, chi < 1 or tol < 1e-13; VP_ENUMERIC: NaN/Inf in the grid).
 * The return value is VP_OK unless the batched launches themselves failed.
 * Call between steps (it uses the group's rank records).  Synchronises the
 * context's stream. */
int vp_group_mps_create(vp_group* g, int count, const vp_layout* layouts, const double* const* f_host,
                        const int* chi, const double* tol, mps_t** out, int* status);
/* Diagnostics of the last vp_group_step: its host wall time (ms), the part
 * spent waiting for the device at the rank reads (ms), the number of those
 * waits and the number of kernels launched (each pointer may be NULL). */
int vp_group_stats(const vp_group* g, double* step_ms, double* wait_ms, int64_t* waits, int64_t* launches);
int vp_group_destroy(vp_group* g);

/* ------------------------------------------------ several species (f_s) */

/* Species s of a multi-species run (Problem Statement: the Vlasov equation of
 * every species, Poisson's equation for the net charge; Methods, "Buneman
 * instability", "Collision Operator").  Units: electron charge magnitude and
 * mass; electrons are q = -1, m = 1. */
typedef struct {
  double q;    /* charge (ions +1, electrons -1) */
  double m;    /* mass (> 0) */
  double nu;   /* Dougherty collision rate (0: collisionless) */
  double u;    /* drift of the Dougherty operator nu d/dv[(v - u) f + vth^2 df/dv] */
  double vth;  /* thermal speed of the Dougherty operator (> 0 when nu > 0) */
} vp_species;

typedef struct vp_multi vp_multi;

/* ns species (1..16) sharing one electric field.  layouts[s] gives species
 * s its own v grid; every layout has the same nx, xmin and xmax (one x
 * grid, one field).  f0[s] (ns device MPS, copied) is species s's initial
 * state on layouts[s].  cfg is that of vp_sim_create, applied to every
 * species; only compression level C1 (cfg->level 0 or 1).  Each RK4 stage
 * computes every species' density rho_s, solves Poisson once for the net
 * density -sum_s q_s rho_s (for electrons alone: rho_e, the one-species
 * equation), and advances species s with the one-species operator whose
 * field term is diag(-q_s/m_s E) (x) D_v, plus nu_s [D_c^v diag(v - u_s) +
 * vth_s^2 D_vv] (zero-gradient v derivatives) when nu_s > 0.  Errors:
 * VP_EINVAL (bad argument, x grids differ, level > 1), VP_ECFL (max |v| dt /
 * dx above 0.6963 for some species), VP_ECUDA, VP_ENOMEM. */
int vp_multi_create(vp_ctx* ctx, int ns, const vp_layout* layouts, const vp_species* species,
                    const vp_config* cfg, const mps_t* const* f0, vp_multi** out);
int vp_multi_destroy(vp_multi* m);
/* Advance nsteps; records[nsteps * ns] (host, or NULL): record n*ns + s is
 * step n of species s -- t, the shared field energy W_E, the species' mass
 * sum f_s dx dv (both of the state at the start of the step), its max bond
 * and truncation error after the step. */
int vp_multi_step(vp_multi* m, int nsteps, vp_record* records);
/* Current state of species s (owned by the run; valid until the next step). */
const mps_t* vp_multi_state(const vp_multi* m, int s);

/* ------------------------------------------------- batching and serving */

/* Many independent runs on one GPU (no counterpart in the paper: the
 * serving/batching layer around its time stepper).  A pool of
 * `max_concurrent` worker threads, each with its own context and CUDA stream;
 * a request is admitted first-in first-out when a worker is free and its
 * footprint fits `mem_budget_bytes`; requests submitted while others run
 * join as slots free up, and the runs' kernels overlap on the device.  Each
 * run's result is independent of what else runs (own buffers and stream). */
typedef struct vp_batch vp_batch;

typedef struct {
  uint64_t id;
  int status;           /* VP_OK or the run's error code */
  int nsteps;
  double queue_ms;      /* submit -> start */
  double run_ms;        /* start -> finish (MPS creation, steps, readback) */
  double step_ms_p50;   /* per-step latency percentiles of this run (host wall time) */
  double step_ms_p99;
  double field_energy;  /* W_E at the start of the last step */
  int max_bond;
} vp_result;

/* Device bytes a run needs (states, pre-compression sums, factorisation
 * workspaces), used for admission. */
size_t vp_footprint_bytes(const vp_layout* layout, const vp_config* cfg);
/* max_concurrent: resident runs at a time (1..64 worker threads; 1..4096 in
 * lockstep mode).  Errors: VP_EINVAL. */
int vp_batch_create(vp_ctx* ctx, int max_concurrent, size_t mem_budget_bytes, vp_batch** out);
/* Lockstep mode (before vp_batch_start; groups = 0 turns it off): instead of
 * one worker thread per run, `groups` workers (1..16), each with its own
 * context and stream, keep their resident runs in a lockstep group
 * (vp_group_*) and advance them all with one group step.  A worker holds runs
 * of one site count at a time (the count of the first run it admits while
 * empty), so runs of one size step together and the groups of different
 * sizes overlap on the device.  Between steps, runs that have finished or
 * failed leave and pending requests join -- first in, first out among those
 * that match the worker's site count -- while at most max_concurrent runs
 * are resident per worker and all footprints fit the budget (continuous
 * batching).  A run's per-step latency is its group's step.  Requests must be
 * eligible for a group (level C1, plain sweeps, FP64 or FP32 contractions,
 * tol >= 1e-13); others end with VP_EINVAL.  Errors: VP_EINVAL, VP_EBUSY
 * (already started). */
int vp_batch_set_lockstep(vp_batch* b, int groups);
/* Copies f0 (host, dense 2^(nx+nv)); keep_f != 0 keeps f(T) for
 * vp_batch_records.  Errors: VP_ECAPACITY (footprint above the budget). */
int vp_batch_submit(vp_batch* b, const vp_layout* layout, const vp_config* cfg, const double* f0_host,
                    int nsteps, int keep_f, uint64_t* id_out);
/* Start the workers (non-blocking); submission stays open. */
int vp_batch_start(vp_batch* b);
/* Block until every submitted run has finished. */
int vp_batch_wait(vp_batch* b);
/* Non-blocking: up to `max` runs finished since the last poll. */
int vp_batch_poll(vp_batch* b, vp_result* out, int max, int* n_out);
/* Per-step records[nsteps], per-step wall times step_ms[nsteps] (host, may be
 * NULL) and f(T) on the grid (host, needs keep_f) of a finished run. */
int vp_batch_records(vp_batch* b, uint64_t id, vp_record* records, double* step_ms, double* fT_host);
/* Kernels launched so far by the batch's worker contexts (diagnostics; the
 * caller's context counts its own launches in vp_kernel_launches).  Read it
 * while the workers are idle: after vp_batch_wait, or once every submitted
 * run has been polled.  0 for NULL or before vp_batch_start. */
int64_t vp_batch_kernel_launches(const vp_batch* b);
int vp_batch_destroy(vp_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* VPMPS_H */
