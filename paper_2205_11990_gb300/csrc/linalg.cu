// FP64 dense linear algebra of the compression sweeps (SI "Canonicalization and
// Compression"): Householder QR, explicit Q, GEMM, one-sided Jacobi SVD and the
// truncation rule of the truncation-error equation (main text, "MPS
// Representation").  All kernels work on one matrix at a time and spread it
// over every SM: FP64 on GB300 issues about two FMAs per SM per clock, so no
// factorisation may sit on a single SM.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include <cooperative_groups.h>
#include <cuda/atomic>

#include "common.cuh"
#include "dw.cuh"

namespace cg = cooperative_groups;

namespace vp {

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; every thread receives the result.  `red` holds kWarps+1.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double t = lane < kWarps ? red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) red[kWarps] = t;
  }
  __syncthreads();
  return red[kWarps];
}

__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

// Grid-wide barrier for cooperative launches: one monotonic 64-bit arrival
// counter, a release add per block and acquire polling (no reset, no
// generation word).  Every block starts from the counter value the previous
// cooperative kernel left in bar_base.  Waits have a clock limit
// (DevStatus::wait_clocks, ~1 s by default): on expiry the block records
// err = 1 and the barrier reports failure, so the kernel returns instead of
// hanging.
struct GridSync {
  DevStatus* st;
  unsigned nb;
  unsigned long long target;
  __device__ GridSync(DevStatus* s, unsigned n) : st(s), nb(n), target(0) {
    if (nb > 1) target = *(volatile unsigned long long*)&st->bar_base;
  }
  __device__ bool sync() {
    __syncthreads();
    if (nb > 1) {
      target += nb;
      if (threadIdx.x == 0) {
        cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> cnt(st->bar_count);
        cnt.fetch_add(1ull, cuda::memory_order_release);
        const long long t0 = clock64(), limit = *(volatile long long*)&st->wait_clocks;
        while (cnt.load(cuda::memory_order_acquire) < target) {
          if (ld_volatile(&st->err) != 0) break;
          if (clock64() - t0 > limit) {
            atomicExch(&st->err, 1);
            break;
          }
        }
      }
      __syncthreads();
    }
    return ld_volatile(&st->err) == 0;
  }
  // Called by every block after its last sync(); block 0 publishes the base.
  __device__ void finish() {
    if (nb > 1 && blockIdx.x == 0 && threadIdx.x == 0) st->bar_base = target;
  }
};

static int coop_launch(vp_ctx* ctx, cudaStream_t stream, const void* fn, int blocks, int threads, void** args,
                       size_t smem, const char* what) {
  ctx->launches++;
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(threads), args, smem, stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, what);
  return VP_OK;
}

// ------------------------------------------------------------ transposition
__global__ void k_to_colmajor(const double* __restrict__ A, int m, int n, double* __restrict__ out) {
  __shared__ double tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int r = by + y, c = bx + threadIdx.x;
    if (r < m && c < n) tile[y][threadIdx.x] = A[(size_t)r * n + c];
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int c = bx + y, r = by + threadIdx.x;
    if (r < m && c < n) out[(size_t)c * m + r] = tile[threadIdx.x][y];
  }
}

int launch_to_colmajor(vp_ctx* ctx, const double* A, int m, int n, double* out) {
  dim3 grid((n + 31) / 32, (m + 31) / 32);
  ctx->launches++;
  k_to_colmajor<<<grid, dim3(32, 8), 0, ctx->stream>>>(A, m, n, out);
  return check_launch(ctx, "to_colmajor");
}

// ------------------------------------------------------------ Householder QR
// Column-cyclic ownership: column k belongs to block k % gridDim.x.  Step j:
// the owner of column j (already updated by H_0..H_{j-1}, which it applied
// itself) forms the reflector H_j = I - tau v v^T (LAPACK dlarfg convention,
// v_j = 1) and publishes v in a double buffer; after one grid barrier every
// block applies H_j to the columns it owns.  One barrier per column.
template <class Sync>
__global__ void __launch_bounds__(kThreads) k_qr_factor(double* A, int m, int n, double* tau,
                                                        double* vbuf, DevStatus* st) {
  __shared__ double red[kWarps + 1];
  const int nb = gridDim.x, bid = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int p = min(m, n);
  Sync gs(st, nb);
  for (int j = 0; j < p; ++j) {
    __syncthreads();
    double* vj = vbuf + (size_t)(j & 1) * m;
    if (bid == j % nb) {
      double* col = A + (size_t)j * m;
      double s = 0.0;
      for (int i = j + 1 + threadIdx.x; i < m; i += kThreads) {
        const double x = col[i];
        s = fma(x, x, s);
      }
      s = block_sum(s, red);
      const double x0 = col[j];
      double t = 0.0, beta = x0, scale = 0.0;
      if (s > 0.0) {
        const double nrm = sqrt(fma(x0, x0, s));
        beta = x0 >= 0.0 ? -nrm : nrm;
        t = (beta - x0) / beta;
        scale = 1.0 / (x0 - beta);
      }
      for (int i = j + 1 + threadIdx.x; i < m; i += kThreads) {
        const double v = col[i] * scale;
        col[i] = v;
        __stcg(vj + i, v);
      }
      if (threadIdx.x == 0) {
        col[j] = beta;
        __stcg(vj + j, 1.0);
        __stcg(tau + j, t);
      }
      __threadfence();
    }
    if (!gs.sync()) return;
    const double t = __ldcg(tau + j);
    if (t == 0.0) continue;
    // first owned column strictly right of j
    const int k0 = (j + 1) + ((bid - (j + 1) % nb) % nb + nb) % nb;
    for (int k = k0 + warp * nb; k < n; k += kWarps * nb) {
      double* col = A + (size_t)k * m;
      double w = 0.0;
      for (int i = j + lane; i < m; i += 32) w = fma(__ldcg(vj + i), col[i], w);
      w = warp_sum(w) * t;
      for (int i = j + lane; i < m; i += 32) col[i] = fma(-w, __ldcg(vj + i), col[i]);
    }
  }
  gs.finish();
}

// Look-ahead QR for the cooperative grid (factors too large for one cluster):
// no grid barrier.  Reflector j is published as double words in V (column j,
// V[j][j] = 1) and T[j] by a release store of a monotonic counter; at step j
// every block waits only for reflector j.  In the owner of column j+1, warp
// 0 applies H_j to that column, forms and publishes reflector j+1 while the
// other warps apply H_j to the rest of the block's columns; the counter base
// carries over between launches (the last block to finish records it).  The
// block's columns are held as double-word values (dw.cuh) in shared memory
// (in global scratch when they do not fit), the arithmetic on the FP32 pipe.
// Column k is scaled by 2^-e_k on load (A D = Q (R D): only R changes, and
// is unscaled on store); each reflector is formed on its column rescaled by
// a further power of two (v and tau do not depend on the scale), so no
// square leaves the FP32 range.  The output A, tau is the FP64 LAPACK layout
// of k_qr_factor.
// nb blocks factor the matrix, this block is number bid of them.
__device__ __forceinline__ void qr_factor_dw_body(double* A, int m, int n, double* tau, dw* V, dw* T, dw* gcols,
                                                  int* gexp, DevStatus* st, const int nb, const int bid) {
  extern __shared__ dw cols_sm[];
  __shared__ int s_ok;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int p = min(m, n);
  const int nown = bid < n ? (n - bid + nb - 1) / nb : 0;
  const int nmax = (n + nb - 1) / nb;
  // the block's columns (and their scale exponents) in shared memory, or in
  // global scratch (gcols, gexp: column k at k m) when they do not fit
  dw* cols = gcols ? gcols + (size_t)bid * m : cols_sm;
  const size_t cstride = gcols ? (size_t)nb * m : (size_t)m;
  int* cexp = gcols ? gexp + bid : reinterpret_cast<int*>(cols_sm + (size_t)nmax * m);
  const int estride = gcols ? nb : 1;
  const unsigned long long base = *(volatile unsigned long long*)&st->pub_base;
  cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> pub(st->pub_count);

  // load the owned columns (k = bid + lc nb), each scaled by a power of two
  for (int lc = warp; lc < nown; lc += kWarps) {
    const double* a = A + (size_t)(bid + lc * nb) * m;
    float mx = 0.f;
    for (int i = lane; i < m; i += 32) mx = fmaxf(mx, fabsf(__double2float_rn(a[i])));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.f) frexpf(mx, &e);
    if (lane == 0) cexp[lc * estride] = e;
    const double sc = ldexp(1.0, -e);
    dw* c = cols + (size_t)lc * cstride;
    for (int i = lane; i < m; i += 32) c[i] = dw_from(a[i] * sc);
  }
  __syncthreads();

  // H_j applied to a local column by one warp: c -= (t (v . c)) v, rows >= j
  auto apply = [&](int j, dw* c) {
    const dw* v = V + (size_t)j * m;
    const float2 t2 = __ldcg(reinterpret_cast<const float2*>(T + j));
    const dw t = {t2.x, t2.y};
    dw_acc acc;
    for (int i = j + lane; i < m; i += 32) {
      const float2 vv = __ldcg(reinterpret_cast<const float2*>(v + i));
      dw_dot_step(acc, {vv.x, vv.y}, c[i]);
    }
    const dw w = dw_mul(dw_warp_sum(dw_acc_value(acc)), t);
    if (w.hi == 0.f) return;
    for (int i = j + lane; i < m; i += 32) {
      const float2 vv = __ldcg(reinterpret_cast<const float2*>(v + i));
      c[i] = dw_add(c[i], dw_neg(dw_mul(w, {vv.x, vv.y})));
    }
  };
  // the critical chain of column j (one warp of its owner): H_{j-1}, then
  // reflector j formed, stored locally and published
  auto critical = [&](int j) {
    dw* c = cols + (size_t)(j / nb) * cstride;
    if (j > 0) apply(j - 1, c);
    __syncwarp();
    float mx = 0.f;
    for (int i = j + lane; i < m; i += 32) mx = fmaxf(mx, fabsf(c[i].hi));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.f) frexpf(mx, &e);
    dw_acc acc;
    for (int i = j + 1 + lane; i < m; i += 32) {
      const dw x = dw_ldexp(c[i], -e);
      dw_dot_step(acc, x, x);
    }
    const dw s = dw_warp_sum(dw_acc_value(acc));
    const dw x0 = dw_ldexp(c[j], -e);
    dw t = {0.f, 0.f}, beta = x0, scale = {0.f, 0.f};
    if (s.hi > 0.f) {
      const dw nrm = dw_sqrt(dw_add(dw_mul(x0, x0), s));
      beta = x0.hi >= 0.f ? dw_neg(nrm) : nrm;
      t = dw_div(dw_add(beta, dw_neg(x0)), beta);
      scale = dw_div({1.0f, 0.0f}, dw_add(x0, dw_neg(beta)));
    }
    dw* v = V + (size_t)j * m;
    for (int i = j + 1 + lane; i < m; i += 32) {
      const dw vi = dw_mul(dw_ldexp(c[i], -e), scale);
      c[i] = vi;
      __stcg(reinterpret_cast<float2*>(v + i), make_float2(vi.hi, vi.lo));
    }
    __syncwarp();
    if (lane == 0) {
      c[j] = dw_ldexp(beta, e);
      __stcg(reinterpret_cast<float2*>(v + j), make_float2(1.0f, 0.0f));
      __stcg(reinterpret_cast<float2*>(T + j), make_float2(t.hi, t.lo));
      tau[j] = dw_to(t);
    }
    __threadfence();
    __syncwarp();
    if (lane == 0) pub.store(base + j + 1, cuda::memory_order_release);
  };
  auto wait = [&](int j) -> bool {
    if (tid == 0) {
      int ok = 1;
      const long long t0 = clock64(), limit = *(volatile long long*)&st->wait_clocks;
      while (pub.load(cuda::memory_order_acquire) < base + j + 1) {
        if (ld_volatile(&st->err) != 0) {
          ok = 0;
          break;
        }
        if (clock64() - t0 > limit) {
          atomicExch(&st->err, 1);
          ok = 0;
          break;
        }
      }
      s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
  };

  if (bid == 0 && warp == 0) critical(0);
  bool ok = true;
  for (int j = 0; j < p; ++j) {
    if (!wait(j)) {
      ok = false;
      break;
    }
    const bool owner = j + 1 < p && bid == (j + 1) % nb;
    if (owner && warp == 0) {
      critical(j + 1);
      continue;
    }
    const int wk = owner ? warp - 1 : warp, nwk = owner ? kWarps - 1 : kWarps;
    // owned columns k >= j + 2: local index lc with bid + lc nb >= j + 2
    const int lc0 = (j + 2 - bid + nb - 1) / nb > 0 ? (j + 2 - bid + nb - 1) / nb : 0;
    for (int lc = lc0 + wk; lc < nown; lc += nwk) apply(j, cols + (size_t)lc * cstride);
  }
  __syncthreads();
  // store: R part unscaled by 2^e_k, reflectors (below the diagonal of the
  // first p columns) as they are
  for (int lc = warp; lc < nown; lc += kWarps) {
    const int k = bid + lc * nb;
    const double sc = ldexp(1.0, cexp[lc * estride]);
    const dw* c = cols + (size_t)lc * cstride;
    double* a = A + (size_t)k * m;
    for (int i = lane; i < m; i += 32) a[i] = (k < p && i > k) ? dw_to(c[i]) : dw_to(c[i]) * sc;
  }
  __syncthreads();
  if (tid == 0 && ok) {
    __threadfence();
    if (atomicAdd(&st->pub_done, 1u) == (unsigned)nb - 1) {
      st->pub_base = base + p;
      st->pub_done = 0u;
      __threadfence();
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_qr_factor_dw(double* A, int m, int n, double* tau, dw* V, dw* T,
                                                          dw* gcols, int* gexp, DevStatus* st) {
  qr_factor_dw_body(A, m, n, tau, V, T, gcols, gexp, st, gridDim.x, blockIdx.x);
}

// Cluster-resident double-word QR (small factors).  Column k lives in CTA
// k % CS (slot k / CS) as double words, scaled by its own power of two as in
// k_qr_factor_dw.  Step j: in the owner of column j+1, warp 0 applies H_j to
// that column, forms reflector j+1 in place and pushes it (rows >= j+1,
// leading 1) with its tau into every CTA's incoming buffer (j+1) % 2 through
// distributed shared memory; the other warps, and every other CTA, apply H_j
// (read from the local incoming buffer j % 2) to their columns right of j+1.
// One hardware cluster barrier per step orders the pushes.
__device__ __forceinline__ void k_qr_factor_cdw_body(double* A, int m, int n, double* tau) {
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int p = min(m, n);
  const int nmax = (n + CS - 1) / CS;
  const int nown = rank < n ? (n - rank + CS - 1) / CS : 0;
  extern __shared__ double qsm_raw[];
  dw* cols = reinterpret_cast<dw*>(qsm_raw);  // nmax columns of m
  dw* vbuf = cols + (size_t)nmax * m;         // 2 x m incoming reflectors
  dw* tbuf = vbuf + 2 * (size_t)m;            // 2 incoming taus
  int* cexp = reinterpret_cast<int*>(tbuf + 2);
  // a one-CTA cluster needs only the block barrier
  auto csync = [&] {
    if (CS == 1)
      __syncthreads();
    else
      cl.sync();
  };

  for (int lc = warp; lc < nown; lc += kWarps) {
    const double* a = A + (size_t)(rank + lc * CS) * m;
    float mx = 0.f;
    for (int i = lane; i < m; i += 32) mx = fmaxf(mx, fabsf(__double2float_rn(a[i])));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.f) frexpf(mx, &e);
    if (lane == 0) cexp[lc] = e;
    const double sc = ldexp(1.0, -e);
    dw* c = cols + (size_t)lc * m;
    for (int i = lane; i < m; i += 32) c[i] = dw_from(a[i] * sc);
  }

  // H_j (from the local incoming buffer) applied to a local column, one warp
  auto apply = [&](int j, dw* c) {
    const dw* v = vbuf + (size_t)(j & 1) * m;
    const dw t = tbuf[j & 1];
    if (t.hi == 0.f) return;
    dw_acc acc;
    for (int i = j + lane; i < m; i += 32) dw_dot_step(acc, v[i], c[i]);
    const dw w = dw_mul(dw_warp_sum(dw_acc_value(acc)), t);
    if (w.hi == 0.f) return;
    for (int i = j + lane; i < m; i += 32) c[i] = dw_add(c[i], dw_neg(dw_mul(w, v[i])));
  };
  // reflector j formed in place in local column c, pushed to every CTA
  auto reflect_push = [&](int j, dw* c) {
    float mx = 0.f;
    for (int i = j + lane; i < m; i += 32) mx = fmaxf(mx, fabsf(c[i].hi));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.f) frexpf(mx, &e);
    dw_acc acc;
    for (int i = j + 1 + lane; i < m; i += 32) {
      const dw x = dw_ldexp(c[i], -e);
      dw_dot_step(acc, x, x);
    }
    const dw s = dw_warp_sum(dw_acc_value(acc));
    const dw x0 = dw_ldexp(c[j], -e);
    dw t = {0.f, 0.f}, beta = x0, scale = {0.f, 0.f};
    if (s.hi > 0.f) {
      const dw nrm = dw_sqrt(dw_add(dw_mul(x0, x0), s));
      beta = x0.hi >= 0.f ? dw_neg(nrm) : nrm;
      t = dw_div(dw_add(beta, dw_neg(x0)), beta);
      scale = dw_div({1.0f, 0.0f}, dw_add(x0, dw_neg(beta)));
    }
    for (int i = j + 1 + lane; i < m; i += 32) c[i] = dw_mul(dw_ldexp(c[i], -e), scale);
    __syncwarp();
    if (lane == 0) {
      c[j] = dw_ldexp(beta, e);
      tau[j] = dw_to(t);
    }
    for (int r = 0; r < CS; ++r) {
      dw* dst = cl.map_shared_rank(vbuf + (size_t)(j & 1) * m, r);
      for (int i = j + lane; i < m; i += 32) dst[i] = (i == j) ? dw{1.0f, 0.0f} : c[i];
      if (lane == 0) *cl.map_shared_rank(tbuf + (j & 1), r) = t;
    }
  };

  csync();  // every CTA resident before the first remote write
  if (rank == 0 && warp == 0 && p > 0) reflect_push(0, cols);
  csync();
  for (int j = 0; j < p; ++j) {
    const bool owner = j + 1 < p && rank == (j + 1) % CS;
    if (owner && warp == 0) {
      dw* c = cols + (size_t)((j + 1) / CS) * m;
      apply(j, c);
      __syncwarp();
      reflect_push(j + 1, c);
    } else {
      const int wk = owner ? warp - 1 : warp, nwk = owner ? kWarps - 1 : kWarps;
      const int lc0 = (j + 2 - rank + CS - 1) / CS > 0 ? (j + 2 - rank + CS - 1) / CS : 0;
      for (int lc = lc0 + wk; lc < nown; lc += nwk) apply(j, cols + (size_t)lc * m);
    }
    csync();
  }
  for (int lc = warp; lc < nown; lc += kWarps) {
    const int k = rank + lc * CS;
    const double sc = ldexp(1.0, cexp[lc]);
    const dw* c = cols + (size_t)lc * m;
    double* a = A + (size_t)k * m;
    for (int i = lane; i < m; i += 32) a[i] = (k < p && i > k) ? dw_to(c[i]) : dw_to(c[i]) * sc;
  }
}
__global__ void __launch_bounds__(kThreads) k_qr_factor_cdw(double* A, int m, int n, double* tau) { k_qr_factor_cdw_body(A, m, n, tau); }

// Cluster-resident double-word QR (factors up to a 16-CTA cluster's shared
// memory).  Column k lives in CTA k % CS (slot k / CS) as double words scaled
// by its own power of two.  Reflector j is formed in its column by the owner,
// which also publishes it through L2: rows > j as double words in A's column
// j, its tau in row j.  Step j: one cluster barrier makes reflector j visible,
// every CTA loads it into its own buffer; then in the owner of column j+1 the
// first CW warps apply H_j to that column and form reflector j+1 in place
// (rows split over the CW warps, partial sums combined in a fixed order
// behind a named barrier), while every other warp applies H_j to the columns
// right of j+1.  A's columns are rewritten with the factor after the last
// barrier.  The L2 copy replaced a pull of each reflector from the owner's
// shared memory through DSMEM, where up to sixteen CTAs wait on one SM's
// DSMEM bandwidth (measured on GB300, two problems per launch: 3.00 -> 2.13 ms
// at 512 x 504 on 16 CTAs, 1.17 -> 0.91 ms at 1008 x 135 on 8, 0.35 -> 0.33 ms
// at 240 x 90; bit-identical results).  The per-row arithmetic is that of
// k_qr_factor_dw; only the order in which the critical column's partial sums
// are added differs.
template <int NT, int CW>
__device__ __forceinline__ void k_qr_factor_cl_body(double* A, int m, int n, double* tau) {
  constexpr int NW = NT / 32;
  static_assert(CW >= 1 && CW < NW, "critical warps must leave bulk warps");
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int p = min(m, n);
  const int nmax = (n + CS - 1) / CS;
  const int nown = rank < n ? (n - rank + CS - 1) / CS : 0;
  extern __shared__ double qsm_raw[];
  dw* cols = reinterpret_cast<dw*>(qsm_raw);  // nmax columns of m
  dw* vin = cols + (size_t)nmax * m;          // reflector of the step (m)
  dw* tsl = vin + m;                          // tau of each owned reflector (nmax)
  dw* tin = tsl + nmax;                       // tau of the step
  int* cexp = reinterpret_cast<int*>(tin + 1);
  __shared__ dw red[3][CW];                   // partial sums of the critical warps
  __shared__ float redm[CW];

  for (int lc = warp; lc < nown; lc += NW) {
    const double* a = A + (size_t)(rank + lc * CS) * m;
    float mx = 0.f;
    for (int i = lane; i < m; i += 32) mx = fmaxf(mx, fabsf(__double2float_rn(a[i])));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.f) frexpf(mx, &e);
    if (lane == 0) cexp[lc] = e;
    const double sc = ldexp(1.0, -e);
    dw* c = cols + (size_t)lc * m;
    for (int i = lane; i < m; i += 32) c[i] = dw_from(a[i] * sc);
  }

  // H_j applied to a bulk column by one warp
  auto apply = [&](int j, dw* c) {
    const dw t = *tin;
    if (t.hi == 0.f) return;
    dw_acc acc;
    dw_dot_rows(acc, vin, c, j, m, lane);
    const dw w = dw_mul(dw_warp_sum(dw_acc_value(acc)), t);
    if (w.hi == 0.f) return;
    dw_axpy_rows(c, vin, w, j, m, lane);
  };
  auto cbar = [] { asm volatile("bar.sync 1, %0;" ::"r"(CW * 32) : "memory"); };
  // Critical warps (warp < CW): H_{j-1} applied to column j (when j > 0),
  // then reflector j formed in place; warp w handles rows i with
  // (i - j) / 32 = w mod CW.
  auto critical = [&](int j, dw* c, int lc) {
    const int r0 = j + 32 * warp + lane, rs = 32 * CW;
    if (j > 0) {  // H_{j-1} acts on rows >= j - 1 (its leading 1 sits in row j - 1)
      const int a0 = r0 - 1;
      const dw t = *tin;
      dw_acc acc;
      for (int i = a0; i < m; i += rs) dw_dot_step(acc, vin[i], c[i]);
      const dw part = dw_warp_sum(dw_acc_value(acc));
      if (lane == 0) red[0][warp] = part;
      cbar();
      dw dot = red[0][0];
      for (int w = 1; w < CW; ++w) dot = dw_add(dot, red[0][w]);
      const dw wv = dw_mul(dot, t);
      if (t.hi != 0.f && wv.hi != 0.f)
        for (int i = a0; i < m; i += rs) c[i] = dw_add(c[i], dw_neg(dw_mul(wv, vin[i])));
    }
    float mx = 0.f;
    for (int i = r0; i < m; i += rs) mx = fmaxf(mx, fabsf(c[i].hi));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) redm[warp] = mx;
    cbar();
    for (int w = 0; w < CW; ++w) mx = fmaxf(mx, redm[w]);
    int e = 0;
    if (mx > 0.f) frexpf(mx, &e);
    const dw x0 = dw_ldexp(c[j], -e);
    dw_acc acc;
    for (int i = r0; i < m; i += rs)
      if (i > j) {
        const dw x = dw_ldexp(c[i], -e);
        dw_dot_step(acc, x, x);
      }
    const dw part = dw_warp_sum(dw_acc_value(acc));
    if (lane == 0) red[1][warp] = part;
    cbar();  // every critical warp has read x0 and its partial sum is in
    dw sq = red[1][0];
    for (int w = 1; w < CW; ++w) sq = dw_add(sq, red[1][w]);
    dw t = {0.f, 0.f}, beta = x0, scale = {0.f, 0.f};
    if (sq.hi > 0.f) {
      const dw nrm = dw_sqrt(dw_add(dw_mul(x0, x0), sq));
      beta = x0.hi >= 0.f ? dw_neg(nrm) : nrm;
      t = dw_div(dw_add(beta, dw_neg(x0)), beta);
      scale = dw_div({1.0f, 0.0f}, dw_add(x0, dw_neg(beta)));
    }
    dw* gj = reinterpret_cast<dw*>(A + (size_t)j * m);
    for (int i = r0; i < m; i += rs)
      if (i > j) {
        const dw v = dw_mul(dw_ldexp(c[i], -e), scale);
        c[i] = v;
        __stcg(reinterpret_cast<float2*>(gj + i), make_float2(v.hi, v.lo));
      }
    if (warp == 0 && lane == 0) {
      c[j] = dw_ldexp(beta, e);
      tsl[lc] = t;
      tau[j] = dw_to(t);
      __stcg(reinterpret_cast<float2*>(gj + j), make_float2(t.hi, t.lo));
    }
  };

  __syncthreads();
  if (rank == 0 && warp < CW && p > 0) critical(0, cols, 0);
  for (int j = 0; j < p; ++j) {
    cl.sync();  // reflector j formed; every CTA done with the previous step
    {
      // every load of the batch issued before any local store
      constexpr int PB = 8;
      const float2* g = reinterpret_cast<const float2*>(A + (size_t)j * m);
      for (int i0 = j + tid; i0 < m; i0 += NT * PB) {
        float2 tmp[PB];
#pragma unroll
        for (int u = 0; u < PB; ++u) {
          const int i = i0 + u * NT;
          if (i < m) tmp[u] = __ldcg(g + i);
        }
#pragma unroll
        for (int u = 0; u < PB; ++u) {
          const int i = i0 + u * NT;
          if (i < m) vin[i] = (i == j) ? dw{1.0f, 0.0f} : dw{tmp[u].x, tmp[u].y};
        }
      }
      if (tid == 0) {
        const float2 tj = __ldcg(g + j);
        *tin = {tj.x, tj.y};
      }
    }
    __syncthreads();
    const bool owner = j + 1 < p && rank == (j + 1) % CS;
    if (owner && warp < CW) {
      const int lc = (j + 1) / CS;
      critical(j + 1, cols + (size_t)lc * m, lc);
    } else {
      const int wk = owner ? warp - CW : warp, nwk = owner ? NW - CW : NW;
      const int lc0 = (j + 2 - rank + CS - 1) / CS > 0 ? (j + 2 - rank + CS - 1) / CS : 0;
      for (int lc = lc0 + wk; lc < nown; lc += nwk) apply(j, cols + (size_t)lc * m);
    }
  }
  cl.sync();  // every CTA is done with every published reflector
  for (int lc = warp; lc < nown; lc += NW) {
    const int k = rank + lc * CS;
    const double sc = ldexp(1.0, cexp[lc]);
    const dw* c = cols + (size_t)lc * m;
    double* a = A + (size_t)k * m;
    for (int i = lane; i < m; i += 32) a[i] = (k < p && i > k) ? dw_to(c[i]) : dw_to(c[i]) * sc;
  }
}
template <int NT, int CW>
__global__ void __launch_bounds__(NT) k_qr_factor_cl(double* A, int m, int n, double* tau) { k_qr_factor_cl_body<NT, CW>(A, m, n, tau); }

static size_t qr_cl_smem(int m, int n, int CS) {
  const size_t nmax = (size_t)(n + CS - 1) / CS;
  return (nmax * m + (size_t)m + nmax + 1) * sizeof(dw) + nmax * sizeof(int);
}

template <int NT, int CW>
static int launch_cl(vp_ctx* ctx, double* A, int m, int n, double* tau, int cs, size_t need) {
  static AttrOnce cattr;
  VP_TRY(cattr.ensure(ctx, (const void*)k_qr_factor_cl<NT, CW>, 200 * 1024, true));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = std::max<size_t>(need, 116 * 1024);  // one CTA of the cluster per SM
  cfg.stream = ctx->stream;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  ctx->launches++;
  VP_CUDA(ctx, cudaLaunchKernelEx(&cfg, k_qr_factor_cl<NT, CW>, A, m, n, tau));
  return VP_OK;
}

int launch_qr_factor_cl(vp_ctx* ctx, double* A, int m, int n, double* tau, int cs) {
  const size_t need = qr_cl_smem(m, n, cs);
  if (need > 200 * 1024) return fail(ctx, VP_ECAPACITY, "qr_factor_cl: factor too large for the cluster");
  return launch_cl<512, 4>(ctx, A, m, n, tau, cs, need);
}

static size_t qr_cdw_smem(int m, int n, int CS) {
  const size_t nmax = (size_t)(n + CS - 1) / CS;
  return (nmax * m + 2 * (size_t)m + 2) * sizeof(dw) + nmax * sizeof(int);
}

// Which kernel factors an m x n matrix.  Measured per column on GB300 (the
// step's shapes): up to ~4e3 elements the small-factor kernel (one CTA up to
// 32 columns, else two; ~2.3 us per column); above, the cluster kernel with
// four critical warps on 16 CTAs (~3-5.5 us per column, against 3.7-17.7 for
// the grid kernel); the grid kernel takes what no cluster's shared memory
// holds.  Factors more
// than twice as wide as tall: the m reflectors depend on the leading m
// columns alone, so that square block (contiguous in the column-major layout)
// is factored in place, Q is formed from its reflectors, and the rest of R is
// one FP64 GEMM, R2 = Q^T A2 (stored as R2^T = A2^T Q, which is A2's
// column-major layout), instead of applying every reflector to all n columns
// one column step at a time.  The choice depends on the shape and the device
// only, so that results do not depend on the context or on the batch.
QRPlan qr_plan(const vp_ctx* ctx, int m, int n) {
  if (std::min(m, n) <= 0) return {QR_NONE, 0};
  if (n > 2 * m && m >= 2) return {QR_WIDE, 0};
  if (ctx->cluster_size > 1 && (long long)m * n <= 4096) {
    // one CTA up to 32 columns, else two (measured on GB300 for 2x2 .. 128x32
    // and 50x50 .. 120x34: four CTAs were never faster; the result does not
    // depend on the CTA count)
    const int cs = n <= 32 ? 1 : 2;
    if (qr_cdw_smem(m, n, cs) <= 200 * 1024) return {QR_CDW, cs};
  }
  if (ctx->cluster_size >= 8 && 2 * m >= n) {
    // the largest cluster: with reflectors published through L2, 16 CTAs beat
    // 8 by 10-21 % on every shape of the step (two problems per launch) and 4
    // were never faster; the result does not depend on the CTA count
    const int cs = ctx->cluster_size >= 16 ? 16 : 8;
    if (qr_cl_smem(m, n, cs) <= 200 * 1024) return {QR_CL, cs};
  }
  return {QR_GRID, 0};
}

// The cooperative grid kernels, for factors beyond a cluster's shared memory:
// enough blocks that each owns a few columns, never more than one per SM.
// st, qrv, qrc: the status words and scratch of the caller (context or batch
// problem).
int qr_factor_grid(vp_ctx* ctx, cudaStream_t stream, DevStatus* st, DevBuf& qrv, DevBuf& qrc, double* A, int m,
                   int n, double* tau, double* vbuf) {
  const int p = std::min(m, n);
  const int cap = ctx->coop_cap > 0 ? std::min(ctx->coop_cap, ctx->num_sms) : ctx->num_sms;
  const int blocks = std::min(cap, std::max(1, n / 2));
  if (blocks > 1) {
    // the same double-word arithmetic whichever the storage, so that the
    // result does not depend on the context's block cap
    const int nmax = (n + blocks - 1) / blocks;
    const size_t smem = (size_t)nmax * m * sizeof(dw) + (size_t)nmax * sizeof(int);
    static AttrOnce qattr;
    VP_TRY(qattr.ensure(ctx, (const void*)k_qr_factor_dw, 200 * 1024, false));
    VP_TRY(reserve(ctx, qrv, (size_t)m * p + p + 8));
    dw* V = reinterpret_cast<dw*>(qrv.p);
    dw* T = V + (size_t)m * p;
    dw* gcols = nullptr;
    int* gexp = nullptr;
    size_t dyn = smem;
    if (smem > 200 * 1024) {
      VP_TRY(reserve(ctx, qrc, (size_t)m * n + n / 2 + 8));
      gcols = reinterpret_cast<dw*>(qrc.p);
      gexp = reinterpret_cast<int*>(gcols + (size_t)m * n);
      dyn = 0;
    }
    void* args[] = {&A, &m, &n, &tau, &V, &T, &gcols, &gexp, &st};
    return coop_launch(ctx, stream, (const void*)k_qr_factor_dw, blocks, kThreads, args, dyn, "qr_factor_dw");
  }
  void* args[] = {&A, &m, &n, &tau, &vbuf, &st};
  return coop_launch(ctx, stream, (const void*)k_qr_factor<GridSync>, blocks, kThreads, args, 0, "qr_factor");
}

int launch_qr_factor(vp_ctx* ctx, double* A, int m, int n, double* tau, double* vbuf) {
  const QRPlan pl = qr_plan(ctx, m, n);
  switch (pl.kind) {
    case QR_NONE:
      return VP_OK;
    case QR_WIDE: {
      VP_TRY(launch_qr_factor(ctx, A, m, m, tau, vbuf));
      VP_TRY(reserve(ctx, ctx->w_wq, (size_t)m * m));
      VP_TRY(launch_qr_formq(ctx, A, m, m, tau, ctx->w_wq.p));
      const size_t rest = (size_t)(n - m) * m;
      VP_TRY(reserve(ctx, ctx->w_wr, rest));
      const int prec = ctx->precision;  // R is part of the factorisation: FP64 in every mode
      ctx->precision = VP_PREC_FP64;
      const int st = launch_gemm(ctx, n - m, m, m, 1.0, A + (size_t)m * m, m, ctx->w_wq.p, m, ctx->w_wr.p, m);
      ctx->precision = prec;
      VP_TRY(st);
      return launch_copy(ctx, ctx->w_wr.p, A + (size_t)m * m, rest);
    }
    case QR_CDW: {
      static AttrOnce cattr;
      VP_TRY(cattr.ensure(ctx, (const void*)k_qr_factor_cdw, 200 * 1024, true));
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      cfg.gridDim = dim3(pl.cs);
      cfg.blockDim = dim3(kThreads);
      cfg.dynamicSmemBytes = std::max<size_t>(qr_cdw_smem(m, n, pl.cs), 116 * 1024);  // one CTA of the cluster per SM
      cfg.stream = ctx->stream;
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = pl.cs;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      ctx->launches++;
      VP_CUDA(ctx, cudaLaunchKernelEx(&cfg, k_qr_factor_cdw, A, m, n, tau));
      return VP_OK;
    }
    case QR_CL:
      return launch_qr_factor_cl(ctx, A, m, n, tau, pl.cs);
    default:
      return qr_factor_grid(ctx, ctx->stream, ctx->status, ctx->w_qrv, ctx->w_qrc, A, m, n, tau, vbuf);
  }
}

// Q = H_0 ... H_{p-1} [I_p; 0] in double words: the reflectors (below the
// diagonal of the factored A, leading 1 implicit) and taus are converted
// once, then one warp per column k of Q applies H_k, ..., H_0 to e_k with
// double-word dot products and updates (each step would otherwise be a chain
// of FP64 FMAs at ~400 cycles apiece); Q is stored row-major (m x p).
__device__ __forceinline__ void k_reflectors_to_dw_body(const double* __restrict__ A, int m, int p, const double* __restrict__ tau,
                                   dw* __restrict__ V, dw* __restrict__ T) {
  const size_t total = (size_t)m * p;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / m), i = (int)(e % m);
    V[e] = i > j ? dw_from(A[e]) : (i == j ? dw{1.0f, 0.0f} : dw{0.0f, 0.0f});
    if (e < (size_t)p) T[e] = dw_from(tau[e]);
  }
}
__global__ void k_reflectors_to_dw(const double* __restrict__ A, int m, int p, const double* __restrict__ tau,
                                   dw* __restrict__ V, dw* __restrict__ T) { k_reflectors_to_dw_body(A, m, p, tau, V, T); }

__device__ __forceinline__ void k_qr_formq_dw_body(const dw* __restrict__ V, int m, int p, const dw* __restrict__ T, dw* __restrict__ scratch,
                              double* __restrict__ Q) {
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (k >= p) return;
  dw* q = scratch + (size_t)k * m;
  for (int i = lane; i < m; i += 32) q[i] = (i == k) ? dw{1.0f, 0.0f} : dw{0.0f, 0.0f};
  __syncwarp();
  for (int j = k; j >= 0; --j) {
    const dw t = T[j];
    if (t.hi == 0.f) continue;
    const dw* v = V + (size_t)j * m;
    dw_acc acc;
    for (int i = j + lane; i < m; i += 32) dw_dot_step(acc, v[i], q[i]);
    const dw w = dw_mul(dw_warp_sum(dw_acc_value(acc)), t);
    for (int i = j + lane; i < m; i += 32) q[i] = dw_add(q[i], dw_neg(dw_mul(w, v[i])));
    __syncwarp();
  }
  for (int i = lane; i < m; i += 32) Q[(size_t)i * p + k] = dw_to(q[i]);
}
__global__ void k_qr_formq_dw(const dw* __restrict__ V, int m, int p, const dw* __restrict__ T, dw* __restrict__ scratch,
                              double* __restrict__ Q) { k_qr_formq_dw_body(V, m, p, T, scratch, Q); }

// The same product with column k of Q held in registers (rows lane + 32 u,
// u < R, for m <= 32 R): per reflector the R reflector entries of a lane are
// loaded together and the dot product and update run on registers, so the
// chain of column k costs one L2 round trip per reflector instead of four.
// Rows above the reflector's start hold zeros in V, which leave the sums and
// the column unchanged.
template <int R>
__device__ __forceinline__ void k_qr_formq_reg_body(const dw* __restrict__ V, int m, int p, const dw* __restrict__ T,
                               double* __restrict__ Q) {
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (k >= p) return;
  dw q[R];
#pragma unroll
  for (int u = 0; u < R; ++u) q[u] = (lane + 32 * u == k) ? dw{1.0f, 0.0f} : dw{0.0f, 0.0f};
  for (int j = k; j >= 0; --j) {
    const float2 t2 = __ldg(reinterpret_cast<const float2*>(T + j));
    if (t2.x == 0.f) continue;
    const dw t = {t2.x, t2.y};
    const dw* v = V + (size_t)j * m;
    dw vv[R];
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const int i = lane + 32 * u;
      if (i < m) {
        const float2 x = __ldg(reinterpret_cast<const float2*>(v + i));
        vv[u] = {x.x, x.y};
      } else {
        vv[u] = {0.f, 0.f};
      }
    }
    dw_acc acc;
#pragma unroll
    for (int u = 0; u < R; ++u) dw_dot_step(acc, vv[u], q[u]);
    const dw w = dw_mul(dw_warp_sum(dw_acc_value(acc)), t);
#pragma unroll
    for (int u = 0; u < R; ++u) q[u] = dw_add(q[u], dw_neg(dw_mul(w, vv[u])));
  }
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const int i = lane + 32 * u;
    if (i < m) Q[(size_t)i * p + k] = dw_to(q[u]);
  }
}
template <int R>
__global__ void k_qr_formq_reg(const dw* __restrict__ V, int m, int p, const dw* __restrict__ T,
                               double* __restrict__ Q) { k_qr_formq_reg_body<R>(V, m, p, T, Q); }

int launch_qr_formq(vp_ctx* ctx, const double* A, int m, int n, const double* tau, double* Q) {
  const int p = std::min(m, n);
  if (p <= 0) return VP_OK;
  VP_TRY(reserve(ctx, ctx->w_q, (size_t)m * p));
  VP_TRY(reserve(ctx, ctx->w_fq, (size_t)m * p + p + 8));
  dw* V = reinterpret_cast<dw*>(ctx->w_fq.p);
  dw* T = V + (size_t)m * p;
  const size_t total = (size_t)m * p;
  const int cb = (int)std::min<size_t>((total + 255) / 256, (size_t)ctx->num_sms * 8);
  ctx->launches += 2;
  k_reflectors_to_dw<<<cb, 256, 0, ctx->stream>>>(A, m, p, tau, V, T);
  VP_TRY(check_launch(ctx, "reflectors_to_dw"));
  if (m <= 512) {  // column of Q in registers
    const int wpb = 4, blocks = (p + wpb - 1) / wpb;
    if (m <= 64) k_qr_formq_reg<2><<<blocks, wpb * 32, 0, ctx->stream>>>(V, m, p, T, Q);
    else if (m <= 128) k_qr_formq_reg<4><<<blocks, wpb * 32, 0, ctx->stream>>>(V, m, p, T, Q);
    else if (m <= 256) k_qr_formq_reg<8><<<blocks, wpb * 32, 0, ctx->stream>>>(V, m, p, T, Q);
    else k_qr_formq_reg<16><<<blocks, wpb * 32, 0, ctx->stream>>>(V, m, p, T, Q);
    return check_launch(ctx, "qr_formq");
  }
  const int wpb = 8;
  k_qr_formq_dw<<<(p + wpb - 1) / wpb, wpb * 32, 0, ctx->stream>>>(V, m, p, T, reinterpret_cast<dw*>(ctx->w_q.p), Q);
  return check_launch(ctx, "qr_formq");
}

__device__ __forceinline__ void k_qr_getr_body(const double* __restrict__ A, int m, int n, int p, double* __restrict__ R) {
  const size_t total = (size_t)p * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / n), k = (int)(e % n);
    R[e] = (j <= k) ? A[(size_t)k * m + j] : 0.0;
  }
}
__global__ void k_qr_getr(const double* __restrict__ A, int m, int n, int p, double* __restrict__ R) { k_qr_getr_body(A, m, n, p, R); }

int launch_qr_getr(vp_ctx* ctx, const double* A, int m, int n, double* R) {
  const int p = std::min(m, n);
  const size_t total = (size_t)p * n;
  if (total == 0) return VP_OK;
  const int blocks = (int)std::min<size_t>((total + 255) / 256, (size_t)ctx->num_sms * 16);
  ctx->launches++;
  k_qr_getr<<<blocks, 256, 0, ctx->stream>>>(A, m, n, p, R);
  return check_launch(ctx, "qr_getr");
}

// ------------------------------------------------------------------- GEMM
// TILE x TILE output tile per block (64 or 32), K step 16, 256 threads with a
// (TILE / 16)^2 register tile each.  FP64 FMA, row-major B and C.  ALoad
// selects the A operand: row-major, or the column-major upper triangle of a
// QR factor.  Each output is the sum over its K slice in ascending k, so the
// tile size does not change the result; the K slicing does (gemm_plan).
// kfirst(row0): the first k that can be nonzero in rows >= row0.
struct ARowMajor {
  const double* A;
  int lda;
  __device__ double operator()(int r, int k) const { return A[(size_t)r * lda + k]; }
  __device__ int kfirst(int) const { return 0; }
};
struct AUpperColMajor {
  const double* A;
  int lda;
  __device__ double operator()(int r, int k) const { return r <= k ? A[(size_t)k * lda + r] : 0.0; }
  __device__ int kfirst(int row0) const { return row0; }  // R[r][k] = 0 for k < r
};

// blockIdx.z selects a K slice of `kslice` columns (split-K); slice s writes
// its partial product to C + s * slice_stride.
// B operand: row-major (K x N), or given as its transpose (N x K row-major).
struct BRowMajor {
  const double* B;
  int ldb;
  __device__ double operator()(int k, int n) const { return B[(size_t)k * ldb + n]; }
};
struct BTransposed {
  const double* B;
  int ldb;
  __device__ double operator()(int k, int n) const { return B[(size_t)n * ldb + k]; }
};

template <class ALoad, class BLoad, class T, int TILE>
__device__ __forceinline__ void gemm_body(int M, int N, int K, double alpha, ALoad a, BLoad bl, double* __restrict__ C,
                                          int ldc, int kslice, size_t slice_stride, int bx, int by, int bz) {
  constexpr int R = TILE / 16;  // outputs per thread along each dimension
  __shared__ T As[16][TILE + 1];
  __shared__ T Bs[16][TILE];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int row0 = bx * TILE, col0 = by * TILE;
  // the terms below the triangle of an upper-triangular A are exact zeros:
  // starting past them leaves every output's sum unchanged
  const int kbeg = max(bz * kslice, a.kfirst(row0)), kend = min(K, bz * kslice + kslice);
  C += bz * slice_stride;
  T acc[R][R] = {};
  for (int k0 = kbeg; k0 < kend; k0 += 16) {
    for (int e = threadIdx.x; e < TILE * 16; e += 256) {
      const int r = e / 16, kk = e % 16;
      const int gr = row0 + r, gk = k0 + kk;
      As[kk][r] = (T)((gr < M && gk < kend) ? a(gr, gk) : 0.0);
    }
    for (int e = threadIdx.x; e < 16 * TILE; e += 256) {
      const int kk = e / TILE, c = e % TILE;
      const int gk = k0 + kk, gc = col0 + c;
      Bs[kk][c] = (T)((gk < kend && gc < N) ? bl(gk, gc) : 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      T av[R], bv[R];
#pragma unroll
      for (int i = 0; i < R; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int i = 0; i < R; ++i) bv[i] = Bs[kk][tx + 16 * i];
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int jj = 0; jj < R; ++jj) acc[i][jj] = fma(av[i], bv[jj], acc[i][jj]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int r = row0 + ty + 16 * i;
    if (r >= M) continue;
#pragma unroll
    for (int jj = 0; jj < R; ++jj) {
      const int c = col0 + tx + 16 * jj;
      if (c < N) C[(size_t)r * ldc + c] = alpha * (double)acc[i][jj];
    }
  }
}

template <class ALoad, class BLoad, class T, int TILE>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, double alpha, ALoad a, BLoad bl,
                                              double* __restrict__ C, int ldc, int kslice, size_t slice_stride) {
  gemm_body<ALoad, BLoad, T, TILE>(M, N, K, alpha, a, bl, C, ldc, kslice, slice_stride, blockIdx.x, blockIdx.y,
                                   blockIdx.z);
}

// How a GEMM is spread over the SMs.  FP64 issues about two FMAs per SM per
// clock on GB300, so a GEMM runs at the rate of the SMs it occupies: 64 x 64
// tiles when they alone give every SM a block, else 32 x 32 tiles, and K
// split into slices (multiples of 16, at most 32) until there are about two
// blocks per SM; the slices' partial products are summed in a fixed order.
// The plan depends on the shape and the device only, so a GEMM gives the same
// bits alone, in a batch or in a group.
GemmPlan gemm_plan(const vp_ctx* ctx, int M, int N, int K) {
  GemmPlan g{64, 1, K};
  const int t64 = ((M + 63) / 64) * ((N + 63) / 64);
  if (t64 >= ctx->num_sms || K <= 16) return g;
  int tiles = t64;
  if (2 * t64 < ctx->num_sms) {
    g.tile = 32;
    tiles = ((M + 31) / 32) * ((N + 31) / 32);
  }
  const int target = 2 * ctx->num_sms;
  if (tiles >= target) return g;
  const int sl = std::min(std::min((target + tiles - 1) / tiles, K / 16), 32);
  if (sl <= 1) return g;
  const int ks = ((K + sl - 1) / sl + 15) / 16 * 16;
  g.kslice = ks;
  g.slices = (K + ks - 1) / ks;
  if (g.slices <= 1) g.kslice = K;
  return g;
}

// Sum of `slices` partial products (fixed order: deterministic).
__device__ __forceinline__ void k_sum_slices_body(const double* __restrict__ P, int M, int N, int slices, size_t stride, double* C,
                             int ldc) {
  const size_t total = (size_t)M * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int s = 0; s < slices; ++s) acc += P[s * stride + e];
    C[(e / N) * ldc + e % N] = acc;
  }
}
__global__ void k_sum_slices(const double* __restrict__ P, int M, int N, int slices, size_t stride, double* C,
                             int ldc) { k_sum_slices_body(P, M, N, slices, stride, C, ldc); }

// The same operands as (row, k) maps for the tensor-core path.
static TcOperand tc_a(const ARowMajor& a) { return {a.A, a.lda, 0}; }
static TcOperand tc_a(const AUpperColMajor& a) { return {a.A, a.lda, 2}; }
static TcOperand tc_b(const BRowMajor& b) { return {b.B, b.ldb, 1}; }
static TcOperand tc_b(const BTransposed& b) { return {b.B, b.ldb, 0}; }

// One GEMM launch (split K per gemm_plan, then the fixed-order slice sum).
template <class ALoad, class BLoad>
static int gemm_dispatch(vp_ctx* ctx, int M, int N, int K, double alpha, ALoad a, BLoad b, double* C, int ldc,
                         const char* what) {
  if (M <= 0 || N <= 0) return VP_OK;
  if (ctx->precision >= VP_PREC_TF32 && K > 0) return launch_tc_gemm(ctx, M, N, K, alpha, tc_a(a), tc_b(b), C, ldc);
  const GemmPlan pl = gemm_plan(ctx, M, N, K);
  dim3 grid((M + pl.tile - 1) / pl.tile, (N + pl.tile - 1) / pl.tile, 1);
  if (grid.y > 65535) return fail(ctx, VP_ECAPACITY, "gemm: N too large");
  // FP32 contraction mode: inputs rounded to FP32, FP32 FMA and accumulation
  const bool f32 = ctx->precision == VP_PREC_FP32_CONTRACT;
  auto kern = pl.tile == 64 ? (f32 ? k_gemm<ALoad, BLoad, float, 64> : k_gemm<ALoad, BLoad, double, 64>)
                            : (f32 ? k_gemm<ALoad, BLoad, float, 32> : k_gemm<ALoad, BLoad, double, 32>);
  int slices = pl.slices;
  const int kslice = pl.kslice;
  if (slices <= 1) {
    ctx->launches++;
    kern<<<grid, 256, 0, ctx->stream>>>(M, N, K, alpha, a, b, C, ldc, K, 0);
    return check_launch(ctx, what);
  }
  const size_t stride = (size_t)M * N;
  VP_TRY(reserve(ctx, ctx->w_split, stride * slices));
  grid.z = slices;
  ctx->launches += 2;
  kern<<<grid, 256, 0, ctx->stream>>>(M, N, K, alpha, a, b, ctx->w_split.p, N, kslice, stride);
  VP_TRY(check_launch(ctx, what));
  const int blocks = (int)std::min<size_t>((stride + 255) / 256, (size_t)ctx->num_sms * 8);
  k_sum_slices<<<blocks, 256, 0, ctx->stream>>>(ctx->w_split.p, M, N, slices, stride, C, ldc);
  return check_launch(ctx, what);
}

int launch_gemm(vp_ctx* ctx, int M, int N, int K, double alpha, const double* A, int lda, const double* B,
                int ldb, double* C, int ldc) {
  return gemm_dispatch(ctx, M, N, K, alpha, ARowMajor{A, lda}, BRowMajor{B, ldb}, C, ldc, "gemm");
}

int launch_gemm_bt(vp_ctx* ctx, int M, int N, int K, const double* A, int lda, const double* Bt, int ldbt, double* C,
                   int ldc) {
  return gemm_dispatch(ctx, M, N, K, 1.0, ARowMajor{A, lda}, BTransposed{Bt, ldbt}, C, ldc, "gemm_bt");
}

int launch_gemm_r(vp_ctx* ctx, int M, int N, int K, const double* Acm, int lda, const double* B, int ldb,
                  double* C, int ldc) {
  return gemm_dispatch(ctx, M, N, K, 1.0, AUpperColMajor{Acm, lda}, BRowMajor{B, ldb}, C, ldc, "gemm_r");
}

// ------------------------------------------------------------ Jacobi SVD
// One-sided (Hestenes) Jacobi on the rows of X: rotate row pairs until all
// are mutually orthogonal; then X = diag(s) V^T and the accumulated rotation
// G (rows of J) gives U = G^T.  Round-robin ("circle") ordering: b' - 1
// rounds of b'/2 disjoint pairs per sweep, one warp per pair, one grid
// barrier per round.
__device__ __forceinline__ int rr_index(int pos, int round, int bp) {
  return pos == 0 ? 0 : 1 + (pos - 1 + round) % (bp - 1);
}

// Plane rotation that zeroes the Gram entry gamma of a row pair with squared
// norms alpha, beta: tan(theta) = t is the smaller root of
// t^2 + 2 t d / gamma - 1 = 0, d = (beta - alpha) / 2, written without the
// quotient d / gamma as t = sign(d) gamma / (|d| + sqrt(d^2 + gamma^2)); then
// cos = 1 / sqrt(1 + t^2), sin = t cos.  Three long-latency operations.
__device__ __forceinline__ void jacobi_rotation(double al, double be, double ga, double& t, double& cs, double& sn) {
  const double d = 0.5 * (be - al);
  t = copysign(1.0, d) * ga / (fabs(d) + sqrt(fma(d, d, ga * ga)));
  cs = rsqrt(fma(t, t, 1.0));
  sn = cs * t;
}

__global__ void __launch_bounds__(kThreads) k_jacobi_rows(double* X, int b, int c, double* J, double eps,
                                                          int max_sweeps, DevStatus* st) {
  const int nb = gridDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gw = blockIdx.x * kWarps + warp, nw = nb * kWarps;
  const int bp = b + (b & 1), npairs = bp / 2, rounds = bp - 1;
  int sweep = 0;
  bool converged = false;
  GridSync gs(st, nb);
  for (; sweep < max_sweeps; ++sweep) {
    unsigned* cnt = &st->rot[sweep % 3];
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&st->rot[(sweep + 1) % 3], 0u);
    for (int round = 0; round < rounds; ++round) {
      for (int pr = gw; pr < npairs; pr += nw) {
        int i = rr_index(pr, round, bp), j = rr_index(bp - 1 - pr, round, bp);
        if (i >= b || j >= b) continue;
        if (i > j) {
          const int t = i;
          i = j;
          j = t;
        }
        double* xi = X + (size_t)i * c;
        double* xj = X + (size_t)j * c;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int q = lane; q < c; q += 32) {
          const double u = __ldcg(xi + q), v = __ldcg(xj + q);
          al = fma(u, u, al);
          be = fma(v, v, be);
          ga = fma(u, v, ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (!(al > 0.0 && be > 0.0)) continue;
        if (!(ga * ga > eps * eps * al * be)) continue;
        double t, cs, sn;
        jacobi_rotation(al, be, ga, t, cs, sn);
        for (int q = lane; q < c; q += 32) {
          const double u = __ldcg(xi + q), v = __ldcg(xj + q);
          __stcg(xi + q, cs * u - sn * v);
          __stcg(xj + q, sn * u + cs * v);
        }
        if (J) {
          double* ji = J + (size_t)i * b;
          double* jj = J + (size_t)j * b;
          for (int q = lane; q < b; q += 32) {
            const double u = __ldcg(ji + q), v = __ldcg(jj + q);
            __stcg(ji + q, cs * u - sn * v);
            __stcg(jj + q, sn * u + cs * v);
          }
        }
        if (lane == 0) atomicAdd(cnt, 1u);
      }
      if (!gs.sync()) return;
    }
    if (__ldcg(cnt) == 0u) {
      converged = true;
      break;
    }
  }
  gs.finish();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->pad2 = sweep + 1;
    if (!converged) atomicCAS(&st->err, 0, 3);
  }
}

// Cluster-resident variant: the b rows of X (length c) and of the rotation
// accumulator J (length b) live in the distributed shared memory of one
// thread-block cluster (row x in CTA x % CS, slot x / CS, X and J parts
// contiguous), one CTA per SM.  A pair is processed by one warp through
// DSMEM pointers; rounds are separated by the hardware cluster barrier
// (about 0.2 us on GB300, against 2 us for a grid-wide software barrier).
__global__ void __launch_bounds__(kThreads) k_jacobi_cluster(double* X, int b, int c, double* J, double eps,
                                                             int max_sweeps, DevStatus* st) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ double sm[];
  const int CS = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int jb = J ? b : 0;  // accumulate the rotations only when J is wanted
  const int rpc = (b + CS - 1) / CS, stride = c + jb;
  double* nrm = sm + (size_t)rpc * stride;                   // squared row norms, one per local row
  unsigned* cnt = reinterpret_cast<unsigned*>(nrm + rpc);
  for (int sl = 0; sl < rpc; ++sl) {
    const int x = sl * CS + rank;
    if (x >= b) break;
    double* row = sm + (size_t)sl * stride;
    for (int q = tid; q < c; q += kThreads) row[q] = X[(size_t)x * c + q];
    for (int q = tid; q < jb; q += kThreads) row[c + q] = (q == x) ? 1.0 : 0.0;
  }
  if (tid < 4) cnt[tid] = 0u;
  unsigned* c0 = cl.map_shared_rank(cnt, 0);
  const int bp = b + (b & 1), npairs = bp / 2, rounds = bp - 1;
  int sweep = 0;
  bool converged = false;
  for (; sweep < max_sweeps; ++sweep) {
    // exact squared norms of the local rows once per sweep; a rotation then
    // updates them as alpha' = alpha - t gamma, beta' = beta + t gamma
    __syncthreads();
    for (int sl = warp; sl < rpc; sl += kWarps) {
      if (sl * CS + rank >= b) break;
      const double* row = sm + (size_t)sl * stride;
      double a = 0.0;
      for (int q = lane; q < c; q += 32) a = fma(row[q], row[q], a);
      a = warp_sum(a);
      if (lane == 0) nrm[sl] = a;
    }
    if (rank == 0 && tid == 0) cnt[(sweep + 1) % 3] = 0u;
    cl.sync();
    unsigned rotated = 0;
    for (int round = 0; round < rounds; ++round) {
      for (int pr = rank + warp * CS; pr < npairs; pr += CS * kWarps) {
        int i = rr_index(pr, round, bp), j = rr_index(bp - 1 - pr, round, bp);
        if (i >= b || j >= b) continue;
        if (i > j) {
          const int t = i;
          i = j;
          j = t;
        }
        double* xi = cl.map_shared_rank(sm + (size_t)(i / CS) * stride, i % CS);
        double* xj = cl.map_shared_rank(sm + (size_t)(j / CS) * stride, j % CS);
        double* ni = cl.map_shared_rank(nrm + i / CS, i % CS);
        double* nj = cl.map_shared_rank(nrm + j / CS, j % CS);
        const double al = *ni, be = *nj;
        double ga = 0.0;
        for (int q = lane; q < c; q += 32) ga = fma(xi[q], xj[q], ga);
        ga = warp_sum(ga);
        if (!(al > 0.0 && be > 0.0)) continue;
        if (!(ga * ga > eps * eps * al * be)) continue;
        double t, cs, sn;
        jacobi_rotation(al, be, ga, t, cs, sn);
        for (int q = lane; q < stride; q += 32) {
          const double u = xi[q], v = xj[q];
          xi[q] = cs * u - sn * v;
          xj[q] = sn * u + cs * v;
        }
        if (lane == 0) {
          *ni = fma(-t, ga, al);
          *nj = fma(t, ga, be);
        }
        ++rotated;
      }
      if (round == rounds - 1 && lane == 0 && rotated) atomicAdd(&c0[sweep % 3], rotated);
      cl.sync();
    }
    if (*(volatile unsigned*)&c0[sweep % 3] == 0u) {
      converged = true;
      break;
    }
  }
  for (int sl = 0; sl < rpc; ++sl) {
    const int x = sl * CS + rank;
    if (x >= b) break;
    const double* row = sm + (size_t)sl * stride;
    for (int q = tid; q < c; q += kThreads) X[(size_t)x * c + q] = row[q];
    for (int q = tid; q < jb; q += kThreads) J[(size_t)x * b + q] = row[c + q];
  }
  if (rank == 0 && tid == 0) {
    st->pad2 = sweep + 1;
    if (!converged) atomicCAS(&st->err, 0, 3);
  }
  cl.sync();  // keep every CTA's shared memory alive until all remote accesses are done
}

__global__ void k_identity(double* J, int b) {
  const size_t total = (size_t)b * b;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x)
    J[e] = (e / b == e % b) ? 1.0 : 0.0;
}

int probe_cluster_size() {
  if (cudaFuncSetAttribute(k_jacobi_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess)
    return 0;
  cudaFuncSetAttribute(k_jacobi_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  for (int cs : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 120 * 1024;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_jacobi_cluster, &cfg) == cudaSuccess && n >= 1) return cs;
    cudaGetLastError();
  }
  return 0;
}

static size_t cluster_jacobi_smem(int b, int c, int CS, bool withJ) {
  const size_t rpc = (size_t)(b + CS - 1) / CS;
  return rpc * (size_t)(c + (withJ ? b : 0) + 1) * sizeof(double) + 4 * sizeof(unsigned);
}

// Block-local variant.  The b rows are split into 2 CS blocks of nb rows (nb
// even, padding rows zero); CTA c of a CS-CTA cluster holds two blocks, "top"
// and "bottom", in its own shared memory.  One block round rotates every
// pair between the two local blocks (nb inner rounds of nb disjoint pairs,
// separated by __syncthreads only); the first block round of a sweep also
// rotates the pairs inside each block.  Then the blocks move on the circle
// schedule (block positions 0..2CS-1, top of CTA c = c, bottom = 2CS-1-c;
// position 0 stays, every other position advances by one), by DSMEM copies
// into the other half of a double buffer and one cluster barrier.  After
// 2CS-1 block rounds every pair of rows has met once (one sweep) and every
// block is back home.
//
// Rotations are applied in scaled form: a row is stored as x~ with a scale
// d (x = d x~), its squared norm alpha kept beside it.  The rotation with
// tan t and cos c becomes x~_i <- x~_i - (t d_j / d_i) x~_j,
// x~_j <- x~_j + (t d_i / d_j) x~_i, d <- c d: two FMAs per element pair
// instead of four operations, with the same rounding bound.  Each sweep
// starts by folding d back into the rows and recomputing alpha exactly.
// Row layout (stride c + jb + 2 doubles): x~ (c), accumulated rotation row
// (jb, when J is wanted), alpha, d.
struct JacBlockCfg {
  int CS, nb, stride;
};

__device__ __forceinline__ int jac_pos_cta(int pos, int CS) { return pos < CS ? pos : 2 * CS - 1 - pos; }
__device__ __forceinline__ int jac_pos_slot(int pos, int CS) { return pos < CS ? 0 : 1; }
__device__ __forceinline__ int jac_next_pos(int pos, int CS) {
  return pos == 0 ? 0 : (pos == 2 * CS - 1 ? 1 : pos + 1);
}

// The pairs of one inner round are processed in three phases, because FP64
// issues at two lanes per clock per SM on GB300 and the scalar work of a
// rotation (threshold, square root, divisions) costs as much as a whole
// 128-element update when every warp repeats it:
//   A  one warp per pair: gamma~ = <x~_i, x~_j> (FMA + warp reduction);
//   B  one lane per pair (warp 0): threshold, rotation, new alpha and d, the
//      two update coefficients;
//   C  one warp per pair: x~_i -= a x~_j, x~_j += b x~_i.
// par[4 p + 0..3]: gamma~, a, b, rotate flag of pair p.
__device__ __forceinline__ void jac_dot(const double* ri, const double* rj, int c, int lane, double* par) {
  double g = 0.0;
  for (int q = lane; q < c; q += 32) g = fma(ri[q], rj[q], g);
  g = warp_sum(g);
  if (lane == 0) par[0] = g;
}

// Returns 1 when the pair is rotated.
__device__ __forceinline__ int jac_params(double* ri, double* rj, int w, double eps2, double* par) {
  double* ei = ri + w;  // alpha, d of row i
  double* ej = rj + w;
  const double al = ei[0], be = ej[0], di = ei[1], dj = ej[1];
  par[3] = 0.0;
  if (!(al > 0.0 && be > 0.0)) return 0;
  const double ga = di * dj * par[0];
  if (!(ga * ga > eps2 * al * be)) return 0;
  double t, cs, sn;
  jacobi_rotation(al, be, ga, t, cs, sn);
  const double inv = 1.0 / (di * dj);
  par[1] = t * dj * dj * inv;
  par[2] = t * di * di * inv;
  par[3] = 1.0;
  ei[0] = fma(-t, ga, al);
  ej[0] = fma(t, ga, be);
  ei[1] = cs * di;
  ej[1] = cs * dj;
  return 1;
}

__device__ __forceinline__ void jac_update(double* ri, double* rj, int w, int lane, const double* par) {
  if (par[3] == 0.0) return;
  const double a = par[1], bb = par[2];
  for (int q = lane; q < w; q += 32) {
    const double u = ri[q], v = rj[q];
    ri[q] = fma(-a, v, u);
    rj[q] = fma(bb, u, v);
  }
}

__global__ void __launch_bounds__(kThreads) k_jacobi_block(double* X, int b, int c, double* J, double eps,
                                                           int max_sweeps, int nb, DevStatus* st) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ double sm[];
  const int CS = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int jb = J ? b : 0;
  const int w = c + jb, stride = w + 2;
  const size_t slot_sz = (size_t)nb * stride;
  // buffer set s, slot (0 top, 1 bottom), row r
  auto row = [&](int s, int slot, int r) { return sm + ((size_t)(s * 2 + slot)) * slot_sz + (size_t)r * stride; };
  double* par = sm + 4 * slot_sz;  // 4 doubles per pair of an inner round
  unsigned* cnt = reinterpret_cast<unsigned*>(par + 4 * nb);
  const double eps2 = eps * eps;
  // one inner round over nb disjoint pairs (rows given by pair_rows)
  auto inner_round = [&](auto pair_rows, unsigned& rotated) {
    for (int pi = warp; pi < nb; pi += kWarps) {
      double *ri, *rj;
      pair_rows(pi, ri, rj);
      jac_dot(ri, rj, c, lane, par + 4 * pi);
    }
    __syncthreads();
    if (warp == 0) {
      for (int pi = lane; pi < nb; pi += 32) {
        double *ri, *rj;
        pair_rows(pi, ri, rj);
        rotated += jac_params(ri, rj, w, eps2, par + 4 * pi);
      }
    }
    __syncthreads();
    for (int pi = warp; pi < nb; pi += kWarps) {
      double *ri, *rj;
      pair_rows(pi, ri, rj);
      jac_update(ri, rj, w, lane, par + 4 * pi);
    }
    __syncthreads();
  };

  // home placement: top = block rank, bottom = block 2 CS - 1 - rank
  for (int slot = 0; slot < 2; ++slot) {
    const int blk = slot == 0 ? rank : 2 * CS - 1 - rank;
    for (int r = 0; r < nb; ++r) {
      const int x = blk * nb + r;
      double* d = row(0, slot, r);
      for (int q = tid; q < stride; q += kThreads) {
        double v = 0.0;
        if (x < b) {
          if (q < c) v = X[(size_t)x * c + q];
          else if (q < w) v = (q - c == x) ? 1.0 : 0.0;
        }
        if (q == w + 1) v = 1.0;  // scale d
        d[q] = v;
      }
    }
  }
  if (tid < 4) cnt[tid] = 0u;
  unsigned* c0 = cl.map_shared_rank(cnt, 0);
  int cur = 0, sweep = 0;
  bool converged = false;
  const int brounds = 2 * CS - 1;
  for (; sweep < max_sweeps; ++sweep) {
    // fold the scales into the rows, exact squared norms
    __syncthreads();
    for (int rr = warp; rr < 2 * nb; rr += kWarps) {
      double* d = row(cur, rr / nb, rr % nb);
      const double sc = d[w + 1];
      double a = 0.0;
      for (int q = lane; q < w; q += 32) {
        const double v = d[q] * sc;
        d[q] = v;
        if (q < c) a = fma(v, v, a);
      }
      a = warp_sum(a);
      __syncwarp();
      if (lane == 0) {
        d[w] = a;
        d[w + 1] = 1.0;
      }
    }
    if (rank == 0 && tid == 0) cnt[(sweep + 1) % 3] = 0u;
    cl.sync();
    unsigned rotated = 0;
    for (int br = 0; br < brounds; ++br) {
      if (br == 0) {
        // pairs inside each local block: round robin over nb rows
        for (int ir = 0; ir < nb - 1; ++ir)
          inner_round(
              [&](int pi, double*& ri, double*& rj) {
                const int slot = pi / (nb / 2), pos = pi % (nb / 2);
                ri = row(cur, slot, rr_index(pos, ir, nb));
                rj = row(cur, slot, rr_index(nb - 1 - pos, ir, nb));
              },
              rotated);
      }
      // pairs between the two local blocks
      for (int s = 0; s < nb; ++s)
        inner_round(
            [&](int pi, double*& ri, double*& rj) {
              ri = row(cur, 0, pi);
              rj = row(cur, 1, (pi + s) % nb);
            },
            rotated);
      if (br == brounds - 1 && warp == 0) {
        const unsigned tot = __reduce_add_sync(0xffffffffu, rotated);
        if (lane == 0 && tot) atomicAdd(&c0[sweep % 3], tot);
      }
      // move both blocks to their next positions (other half of the buffer)
      if (CS > 1) {
        for (int slot = 0; slot < 2; ++slot) {
          const int pos = slot == 0 ? rank : 2 * CS - 1 - rank;
          const int np = jac_next_pos(pos, CS);
          double* dst = cl.map_shared_rank(row(cur ^ 1, jac_pos_slot(np, CS), 0), jac_pos_cta(np, CS));
          const double* src = row(cur, slot, 0);
          for (size_t e = tid; e < slot_sz; e += kThreads) dst[e] = src[e];
        }
        cur ^= 1;
      }
      cl.sync();
    }
    if (*(volatile unsigned*)&c0[sweep % 3] == 0u) {
      converged = true;
      break;
    }
  }
  // blocks are home after a whole number of sweeps: write back x = d x~
  __syncthreads();
  for (int slot = 0; slot < 2; ++slot) {
    const int blk = slot == 0 ? rank : 2 * CS - 1 - rank;
    for (int r = 0; r < nb; ++r) {
      const int x = blk * nb + r;
      if (x >= b) continue;
      const double* d = row(cur, slot, r);
      const double sc = d[w + 1];
      for (int q = tid; q < c; q += kThreads) X[(size_t)x * c + q] = sc * d[q];
      for (int q = tid; q < jb; q += kThreads) J[(size_t)x * b + q] = sc * d[c + q];
    }
  }
  if (rank == 0 && tid == 0) {
    st->pad2 = sweep + 1;
    if (!converged) atomicCAS(&st->err, 0, 3);
  }
  cl.sync();  // keep every CTA's shared memory alive until all remote accesses are done
}

// Double-word variant of k_jacobi_block (the production path): the same
// block-local circle schedule, with the rows held as double-word FP32 pairs
// (dw.cuh), so that the dot products, rotation parameters and updates run on
// the FP32 pipe.  The matrix is first scaled by a power of two common to the
// whole cluster (exact) so that its largest entry is ~1; rows whose squared
// norm falls below 1e-30 of that (singular values under 1e-15 of the
// largest) are left alone.  A rotation uses the standard form
// x_i <- c x_i - s x_j, x_j <- s x_i + c x_j with c = 1/sqrt(1 + t^2) and
// s = c t computed to double-word accuracy from an FP32 tangent t: the angle
// need not be the exact Jacobi angle, the rotation is orthogonal to ~1e-14
// either way.  Pairs rotate while |gamma| > eps sqrt(alpha beta) with eps
// above the ~1e-14 noise of a double-word dot product.  Row layout (stride
// w + 1, w = c + jb, in double-word units): x (c), rotation row (jb), alpha.
__device__ __forceinline__ void k_jacobi_dw_body(double* X, int b, int c, double* J, float eps,
                                                        int max_sweeps, int nb, DevStatus* st) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ double smd[];
  dw* sm = reinterpret_cast<dw*>(smd);
  const int CS = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int jb = J ? b : 0;
  const int w = c + jb, stride = w + 1;
  const size_t slot_sz = (size_t)nb * stride;
  auto row = [&](int s, int slot, int r) { return sm + ((size_t)(s * 2 + slot)) * slot_sz + (size_t)r * stride; };
  dw* par = sm + 4 * slot_sz;  // per pair: flag, cos, sin
  float* red = reinterpret_cast<float*>(par + 3 * nb);  // kWarps + 1 floats
  unsigned* cnt = reinterpret_cast<unsigned*>(red + kWarps + 2);

  // common power-of-two scale: largest |x| over the cluster's rows
  float mx = 0.f;
  for (int slot = 0; slot < 2; ++slot) {
    const int blk = slot == 0 ? rank : 2 * CS - 1 - rank;
    for (int r = 0; r < nb; ++r) {
      const int x = blk * nb + r;
      if (x >= b) continue;
      for (int q = tid; q < c; q += kThreads) mx = fmaxf(mx, fabsf(__double2float_rn(X[(size_t)x * c + q])));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) red[warp] = mx;
  __syncthreads();
  if (tid == 0) {
    float m = 0.f;
    for (int i = 0; i < kWarps; ++i) m = fmaxf(m, red[i]);
    red[kWarps] = m;
  }
  if (tid < 4) cnt[tid] = 0u;
  cl.sync();
  float gmax = 0.f;
  for (int r = 0; r < CS; ++r) gmax = fmaxf(gmax, *cl.map_shared_rank(red + kWarps, r));
  int ex = 0;
  if (gmax > 0.f) frexpf(gmax, &ex);
  const double sc = ldexp(1.0, -ex), inv_sc = ldexp(1.0, ex);

  // home placement: top = block rank, bottom = block 2 CS - 1 - rank
  for (int slot = 0; slot < 2; ++slot) {
    const int blk = slot == 0 ? rank : 2 * CS - 1 - rank;
    for (int r = 0; r < nb; ++r) {
      const int x = blk * nb + r;
      dw* d = row(0, slot, r);
      for (int q = tid; q < stride; q += kThreads) {
        dw v = {0.f, 0.f};
        if (x < b) {
          if (q < c) v = dw_from(X[(size_t)x * c + q] * sc);
          else if (q < w) v.hi = (q - c == x) ? 1.0f : 0.0f;
        }
        d[q] = v;
      }
    }
  }
  unsigned* c0 = cl.map_shared_rank(cnt, 0);
  const float tiny = 1e-30f;

  // Rotation parameters of one pair from gamma = <x_i, x_j> and the squared
  // norms alpha, beta held after each row (false: the pair is left alone).
  auto pair_params = [&](dw al, dw be, dw g, dw& cs, dw& sn, dw& tg) -> bool {
    if (!(al.hi > tiny && be.hi > tiny && fabsf(g.hi) * rsqrtf(al.hi) * rsqrtf(be.hi) > eps)) return false;
    // tangent in FP32 after an exact power-of-two scaling of d and gamma
    // (their squares would leave the FP32 range for small rows)
    const float d0 = 0.5f * dw_add(be, dw_neg(al)).hi;
    int e2;
    frexpf(fmaxf(fabsf(d0), fabsf(g.hi)), &e2);
    const float d = ldexpf(d0, -e2), gs = ldexpf(g.hi, -e2);
    const float t = copysignf(1.0f, d) * gs / (fabsf(d) + sqrtf(fmaf(d, d, gs * gs)));
    if (t == 0.f) return false;
    const dw t2 = two_prod(t, t);
    cs = dw_rsqrt(dw_add({1.0f, 0.0f}, t2));
    sn = dw_mul_f(cs, t);
    tg = dw_mul_f(g, t);
    return true;
  };
  // One inner round over nb disjoint pairs.  With at most one pair per warp
  // (nb <= kWarps, the usual case) pair i belongs to the wpp = kWarps / nb
  // warps i wpp .. i wpp + wpp - 1: each of them forms gamma and the
  // rotation itself (the same operations, so the same bits), and rotates its
  // share of the columns; one named barrier of the pair's warps orders the
  // reads of alpha and beta before their update, and one block barrier ends
  // the round.  With more pairs than warps the round runs in three phases:
  // A dot products (a warp per pair), B rotation parameters (a lane per
  // pair), C updates (a warp per pair), each ended by a block barrier.
  auto inner_round = [&](auto pair_rows, unsigned& rotated) {
    if (nb <= kWarps) {
      const int wpp = kWarps / nb, pi = warp / wpp, part = warp % wpp;
      if (pi < nb) {
        dw *ri, *rj;
        pair_rows(pi, ri, rj);
        dw_acc acc;
        dw_dot_rows(acc, ri, rj, 0, c, lane);
        const dw g = dw_warp_sum(dw_acc_value(acc));
        const dw al = ri[w], be = rj[w];
        dw cs, sn, tg;
        const bool rot = pair_params(al, be, g, cs, sn, tg);
        // every warp of the pair has read alpha and beta before they change
        if (wpp > 1)
          asm volatile("bar.sync %0, %1;" ::"r"(1 + pi), "r"(32 * wpp) : "memory");
        else
          __syncwarp();
        if (rot) {
          if (part == 0 && lane == 0) {
            ri[w] = dw_add(al, dw_neg(tg));
            rj[w] = dw_add(be, tg);
            ++rotated;
          }
          const int span = (w + wpp - 1) / wpp, q0 = part * span;
          if (q0 < w) dw_rot_rows(ri + q0, rj + q0, cs, sn, min(span, w - q0), lane);
        }
      }
      __syncthreads();
      return;
    }
    for (int pi = warp; pi < nb; pi += kWarps) {
      dw *ri, *rj;
      pair_rows(pi, ri, rj);
      dw_acc acc;
      dw_dot_rows(acc, ri, rj, 0, c, lane);
      const dw g = dw_warp_sum(dw_acc_value(acc));
      if (lane == 0) par[3 * pi] = g;
    }
    __syncthreads();
    if (warp == 0) {
      for (int pi = lane; pi < nb; pi += 32) {
        dw *ri, *rj;
        pair_rows(pi, ri, rj);
        const dw al = ri[w], be = rj[w];
        dw cs, sn, tg;
        float flag = 0.f;
        if (pair_params(al, be, par[3 * pi], cs, sn, tg)) {
          ri[w] = dw_add(al, dw_neg(tg));
          rj[w] = dw_add(be, tg);
          par[3 * pi + 1] = cs;
          par[3 * pi + 2] = sn;
          flag = 1.f;
          ++rotated;
        }
        par[3 * pi].hi = flag;
      }
    }
    __syncthreads();
    for (int pi = warp; pi < nb; pi += kWarps) {
      if (par[3 * pi].hi == 0.f) continue;
      dw *ri, *rj;
      pair_rows(pi, ri, rj);
      dw_rot_rows(ri, rj, par[3 * pi + 1], par[3 * pi + 2], w, lane);
    }
    __syncthreads();
  };

  // A pair that would rotate, counted without rotating (the test of
  // inner_round on the same operands in the same order).
  auto dry_pair = [&](const dw* ri, const dw* rj, unsigned& would) {
    dw_acc acc;
    dw_dot_rows(acc, ri, rj, 0, c, lane);
    const dw g = dw_warp_sum(dw_acc_value(acc));
    dw cs, sn, tg;
    if (pair_params(ri[w], rj[w], g, cs, sn, tg) && lane == 0) ++would;
  };

  // Sweeps of the circle schedule until one rotates nothing.  After a sweep
  // with few rotations (at most max(4, b/2)) the next pass is a dry sweep:
  // every pair of the schedule is tested in the same order and orientation
  // but nothing is rotated, so its pairs need no barriers between rounds.  If
  // no pair would rotate, the plain sweep would have rotated nothing either
  // (its operands never change) and the rows are final; otherwise nothing has
  // changed and the plain sweep runs.  The result is the plain schedule's,
  // bit for bit, without its last, rotation-free sweep.
  int cur = 0, iter = 0, sweeps = 0;
  bool converged = false, dry_failed = false;
  unsigned last_rot = 0xffffffffu;
  const unsigned dry_max = (unsigned)max(4, b / 2);
  const int brounds = 2 * CS - 1;
  for (; sweeps < max_sweeps; ++iter) {
    const bool dry = last_rot <= dry_max && !dry_failed;
    // exact squared norms of the local rows
    __syncthreads();
    for (int rr = warp; rr < 2 * nb; rr += kWarps) {
      dw* d = row(cur, rr / nb, rr % nb);
      dw_acc acc;
      dw_dot_rows(acc, d, d, 0, c, lane);
      const dw a = dw_warp_sum(dw_acc_value(acc));
      if (lane == 0) d[w] = a;
    }
    if (rank == 0 && tid == 0) cnt[(iter + 1) % 3] = 0u;
    cl.sync();
    unsigned rotated = 0;
    for (int br = 0; br < brounds; ++br) {
      if (dry) {
        if (br == 0)
          for (int e = warp; e < (nb - 1) * nb; e += kWarps) {
            const int ir = e / nb, pi = e % nb;
            const int slot = pi / (nb / 2), pos = pi % (nb / 2);
            dry_pair(row(cur, slot, rr_index(pos, ir, nb)), row(cur, slot, rr_index(nb - 1 - pos, ir, nb)), rotated);
          }
        for (int e = warp; e < nb * nb; e += kWarps) {
          const int sh = e / nb, pi = e % nb;
          dry_pair(row(cur, 0, pi), row(cur, 1, (pi + sh) % nb), rotated);
        }
      } else {
        if (br == 0) {
          for (int ir = 0; ir < nb - 1; ++ir)
            inner_round(
                [&](int pi, dw*& ri, dw*& rj) {
                  const int slot = pi / (nb / 2), pos = pi % (nb / 2);
                  ri = row(cur, slot, rr_index(pos, ir, nb));
                  rj = row(cur, slot, rr_index(nb - 1 - pos, ir, nb));
                },
                rotated);
        }
        for (int sh = 0; sh < nb; ++sh)
          inner_round(
              [&](int pi, dw*& ri, dw*& rj) {
                ri = row(cur, 0, pi);
                rj = row(cur, 1, (pi + sh) % nb);
              },
              rotated);
      }
      if (br == brounds - 1) {
        const unsigned tot = __reduce_add_sync(0xffffffffu, rotated);
        if (lane == 0 && tot) atomicAdd(&c0[iter % 3], tot);
      }
      if (CS > 1) {
        for (int slot = 0; slot < 2; ++slot) {
          const int pos = slot == 0 ? rank : 2 * CS - 1 - rank;
          const int np = jac_next_pos(pos, CS);
          dw* dst = cl.map_shared_rank(row(cur ^ 1, jac_pos_slot(np, CS), 0), jac_pos_cta(np, CS));
          const dw* src = row(cur, slot, 0);
          for (size_t e = tid; e < slot_sz; e += kThreads) dst[e] = src[e];
        }
        cur ^= 1;
      }
      cl.sync();
    }
    const unsigned tot = *(volatile unsigned*)&c0[iter % 3];
    if (tot == 0u) {
      converged = true;
      ++sweeps;
      break;
    }
    dry_failed = dry;
    if (!dry) {
      ++sweeps;
      last_rot = tot;
    }
  }
  __syncthreads();
  for (int slot = 0; slot < 2; ++slot) {
    const int blk = slot == 0 ? rank : 2 * CS - 1 - rank;
    for (int r = 0; r < nb; ++r) {
      const int x = blk * nb + r;
      if (x >= b) continue;
      const dw* d = row(cur, slot, r);
      for (int q = tid; q < c; q += kThreads) X[(size_t)x * c + q] = dw_to(d[q]) * inv_sc;
      for (int q = tid; q < jb; q += kThreads) J[(size_t)x * b + q] = dw_to(d[c + q]);
    }
  }
  if (rank == 0 && tid == 0) {
    st->pad2 = converged ? sweeps : max_sweeps + 1;  // as the plain schedule counts them
    if (!converged) atomicCAS(&st->err, 0, 3);
  }
  cl.sync();  // keep every CTA's shared memory alive until all remote accesses are done
}
__global__ void __launch_bounds__(kThreads) k_jacobi_dw(double* X, int b, int c, double* J, float eps,
                                                        int max_sweeps, int nb, DevStatus* st) { k_jacobi_dw_body(X, b, c, J, eps, max_sweeps, nb, st); }

static JacBlockCfg jac_block_cfg(int b, int c, bool withJ, int cs_max) {
  JacBlockCfg g{1, 2, 0};
  int cs = 1;
  while (cs < 16 && cs < cs_max && cs * 8 < b) cs *= 2;
  int nb = (b + 2 * cs - 1) / (2 * cs);
  nb += nb & 1;
  if (nb < 2) nb = 2;
  g.CS = cs;
  g.nb = nb;
  g.stride = c + (withJ ? b : 0) + 2;
  return g;
}

static size_t jac_dw_smem(const JacBlockCfg& g) {
  // rows (stride - 1 double words: no scale slot), pair parameters, reduction, counters
  return (4 * (size_t)g.nb * (g.stride - 1) + 3 * (size_t)g.nb) * sizeof(dw) + (kWarps + 2) * sizeof(float) +
         4 * sizeof(unsigned);
}

static size_t jac_block_smem(const JacBlockCfg& g) {
  return (4 * (size_t)g.nb * g.stride + 4 * (size_t)g.nb) * sizeof(double) + 4 * sizeof(unsigned);
}

int jacobi_rows_on(vp_ctx* ctx, cudaStream_t stream, DevStatus* status, double* X, int b, int c, double* J,
                   bool floor_ok) {
  if (b <= 0) return VP_OK;
  const int CS = ctx->cluster_size;
  const JacBlockCfg bc = jac_block_cfg(b, c, J != nullptr, std::max(1, CS));
  if (floor_ok && b > 1 && jac_dw_smem(bc) <= 200 * 1024) {
    static AttrOnce dattr_done;
    VP_TRY(dattr_done.ensure(ctx, (const void*)k_jacobi_dw, 200 * 1024, true));
    const size_t smem = std::max<size_t>(jac_dw_smem(bc), 120 * 1024);
    // rotate while |gamma| > eps sqrt(alpha beta); eps above the double-word
    // dot-product noise, which grows like sqrt(c) u^2
    float eps = (float)(4e-13 * std::sqrt((double)c));
    int max_sweeps = 60;
    int nb = bc.nb;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    cfg.gridDim = dim3(bc.CS);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = bc.CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    ctx->launches++;
    VP_CUDA(ctx, cudaLaunchKernelEx(&cfg, k_jacobi_dw, X, b, c, J, eps, max_sweeps, nb, status));
    return VP_OK;
  }
  if (b > 1 && jac_block_smem(bc) <= 200 * 1024) {
    static AttrOnce battr_done;
    VP_TRY(battr_done.ensure(ctx, (const void*)k_jacobi_block, 200 * 1024, true));
    // one CTA per SM: the FP64 pipe of each SM is the limit
    const size_t smem = std::max<size_t>(jac_block_smem(bc), 120 * 1024);
    double eps = 1e-15 * std::sqrt((double)c);
    int max_sweeps = 60;
    int nb = bc.nb;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    cfg.gridDim = dim3(bc.CS);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = bc.CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    ctx->launches++;
    VP_CUDA(ctx, cudaLaunchKernelEx(&cfg, k_jacobi_block, X, b, c, J, eps, max_sweeps, nb, status));
    return VP_OK;
  }
  if (CS > 0 && b > 1 && cluster_jacobi_smem(b, c, CS, J != nullptr) <= 200 * 1024) {
    static AttrOnce attr_done;
    // at least 120 KB per CTA, so no two CTAs of the cluster share an SM
    const size_t smem = std::max<size_t>(cluster_jacobi_smem(b, c, CS, J != nullptr), 120 * 1024);
    VP_TRY(attr_done.ensure(ctx, (const void*)k_jacobi_cluster, 200 * 1024, true));
    double eps = 1e-15 * std::sqrt((double)c);
    int max_sweeps = 60;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    cfg.gridDim = dim3(CS);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    ctx->launches++;
    VP_CUDA(ctx, cudaLaunchKernelEx(&cfg, k_jacobi_cluster, X, b, c, J, eps, max_sweeps, status));
    return VP_OK;
  }
  if (J) {
    ctx->launches++;
    k_identity<<<std::min(1024, (b * b + 255) / 256 + 1), 256, 0, stream>>>(J, b);
    VP_TRY(check_launch(ctx, "identity"));
  }
  if (b == 1) return VP_OK;
  const int npairs = (b + 1) / 2;
  int blocks = std::min(ctx->num_sms, std::max(1, (npairs + kWarps - 1) / kWarps));
  if ((long long)b * c < 4096) blocks = 1;
  // rotate while |<x_i,x_j>| > eps |x_i||x_j|; eps grows with the dot length
  double eps = 1e-15 * std::sqrt((double)c);
  int max_sweeps = 60;
  DevStatus* st = status;
  void* args[] = {&X, &b, &c, &J, &eps, &max_sweeps, &st};
  return coop_launch(ctx, stream, (const void*)k_jacobi_rows, blocks, kThreads, args, 0, "jacobi_rows");
}

int launch_jacobi_rows(vp_ctx* ctx, double* X, int b, int c, double* J, bool floor_ok) {
  return jacobi_rows_on(ctx, ctx->stream, ctx->status, X, b, c, J, floor_ok);
}

// ------------------------------------------------------------ truncation
// Descending order with ties broken by index, as a strict total order even
// when values are NaN (NaNs first, by index): the rank of each element is
// then a permutation, so the indices written from it always stay in range.
__device__ __forceinline__ bool sorts_before(double a, int ia, double b, int ib) {
  const bool na = isnan(a), nb = isnan(b);
  if (na || nb) return na && (!nb || ia < ib);
  return a > b || (a == b && ia < ib);
}

// Single block: row norms, descending order (ties by index), kept rank by the
// rule r = min(chi, r_tol), r_tol the smallest r with sqrt(sum_{i>=r} s_i^2)
// <= tol ||s|| (tol = 0: keep all), moved down to the start of a cluster of
// values within a relative 1e-5.  A dependent FP64 operation costs hundreds of
// cycles on GB300, so nothing here runs as a serial chain over the values:
// four rows per warp at a time for the norms (each row summed in the same
// order as alone), the tail sums as a block-wide suffix scan (chunk sums,
// then a scan of the chunk totals), r_tol as a minimum over the rows that
// meet the tolerance, and the entanglement entropy as a fixed-order tree sum.
__device__ __forceinline__ void k_select_body(const double* __restrict__ X, int b, int c, int chi, double tol, int* perm,
                         double* sigma, int* d_rank, double* d_err, DevStatus* st) {
  extern __shared__ double sm[];
  double* s = sm;          // b
  double* tail = sm + b;   // b + 1
  __shared__ double ctot[1024];  // per-thread chunk totals, then their suffix sums
  __shared__ double wpart[32];
  __shared__ int rmin, rkeep;
  const int T = blockDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = T >> 5;
  constexpr int RB = 4;
  for (int i0 = warp * RB; i0 < b; i0 += nwarps * RB) {
    double a[RB];
#pragma unroll
    for (int u = 0; u < RB; ++u) a[u] = 0.0;
    for (int q = lane; q < c; q += 32)
#pragma unroll
      for (int u = 0; u < RB; ++u)
        if (i0 + u < b) {
          const double x = X[(size_t)(i0 + u) * c + q];
          a[u] = fma(x, x, a[u]);
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int u = 0; u < RB; ++u) a[u] += __shfl_xor_sync(0xffffffffu, a[u], o);
    if (lane == 0)
#pragma unroll
      for (int u = 0; u < RB; ++u)
        if (i0 + u < b) s[i0 + u] = sqrt(a[u]);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < b; i += T) {
    const double si = s[i];
    if (!isfinite(si)) atomicCAS(&st->err, 0, 2);
    int pos = 0;
    for (int j = 0; j < b; ++j) pos += sorts_before(s[j], j, si, i);
    perm[pos] = i;
    sigma[pos] = si;
  }
  __syncthreads();
  // tail[i] = sum_{k >= i} sigma_k^2: each thread a chunk of k consecutive
  // values (summed smallest first), then a suffix scan of the chunk totals
  const int k = (b + T - 1) / T;
  const int lo = threadIdx.x * k, hi = min(b, lo + k);
  double acc = 0.0;
  for (int i = hi - 1; i >= lo; --i) {
    acc = fma(sigma[i], sigma[i], acc);
    tail[i] = acc;
  }
  ctot[threadIdx.x] = acc;
  if (threadIdx.x == 0) {
    tail[b] = 0.0;
    rmin = b;
  }
  __syncthreads();
  for (int off = 1; off < T; off <<= 1) {
    const double v = ctot[threadIdx.x] + (threadIdx.x + off < T ? ctot[threadIdx.x + off] : 0.0);
    __syncthreads();
    ctot[threadIdx.x] = v;
    __syncthreads();
  }
  const double after = threadIdx.x + 1 < T ? ctot[threadIdx.x + 1] : 0.0;
  for (int i = lo; i < hi; ++i) tail[i] += after;
  __syncthreads();
  const double nrm2 = tail[0];
  if (nrm2 > 0.0 && tol > 0.0) {
    const double thr2 = tol * tol * nrm2;
    for (int q = threadIdx.x + 1; q <= b; q += T)
      if (tail[q] <= thr2) atomicMin(&rmin, q);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int r = 1;
    double err = 0.0;
    if (nrm2 > 0.0) {
      r = min(min(chi, rmin), b);
      while (r > 1 && r < b && (sigma[r - 1] - sigma[r]) <= 1e-5 * sigma[r - 1]) --r;
      if (r < 1) r = 1;
      err = sqrt(tail[r] / nrm2);
    }
    rkeep = r;
    *d_rank = r;
    d_err[0] = err;
  }
  __syncthreads();
  // entanglement entropy of the kept values (main text, EE equation):
  // -sum p log2 p with p_i = s_i^2 / sum_{kept} s^2
  const int r = rkeep;
  const double kept2 = tail[0] - tail[r];
  double ee = 0.0;
  if (kept2 > 0.0)
    for (int q = threadIdx.x; q < r; q += T) {
      const double pq = sigma[q] * sigma[q] / kept2;
      if (pq > 0.0) ee -= pq * log2(pq);
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ee += __shfl_xor_sync(0xffffffffu, ee, o);
  if (lane == 0) wpart[warp] = ee;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < nwarps; ++w) tot += wpart[w];
    d_err[1] = tot;
  }
}
__global__ void k_select(const double* __restrict__ X, int b, int c, int chi, double tol, int* perm,
                         double* sigma, int* d_rank, double* d_err, DevStatus* st) { k_select_body(X, b, c, chi, tol, perm, sigma, d_rank, d_err, st); }

int launch_select(vp_ctx* ctx, const double* X, int b, int c, int chi, double tol, int* perm, double* sigma,
                  int* d_rank, double* d_err) {
  const size_t smem = (size_t)(2 * b + 1) * sizeof(double);
  if (smem > 200 * 1024) return fail(ctx, VP_ECAPACITY, "select: bond too large");
  // always: the kernel's own 8 KB of static shared memory counts against the
  // 48 KB a block gets without the opt-in
  static AttrOnce sattr;
  VP_TRY(sattr.ensure(ctx, (const void*)k_select, 200 * 1024, false));
  ctx->launches++;
  k_select<<<1, 512, smem, ctx->stream>>>(X, b, c, chi, tol, perm, sigma, d_rank, d_err, ctx->status);
  return check_launch(ctx, "select");
}

__device__ __forceinline__ void k_svd_outputs_body(const double* __restrict__ X, const double* __restrict__ J, int b, int c, int r,
                              const int* __restrict__ perm, const double* __restrict__ sigma, double* Vt,
                              double* W) {
  const size_t nv = (size_t)r * c, nw = J ? (size_t)b * r : 0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nv + nw; e += (size_t)gridDim.x * blockDim.x) {
    if (e < nv) {
      const int t = (int)(e / c), q = (int)(e % c);
      const double s = sigma[t];
      Vt[e] = s > 0.0 ? X[(size_t)perm[t] * c + q] / s : 0.0;
    } else {
      const size_t f = e - nv;
      const int i = (int)(f / r), t = (int)(f % r);
      W[f] = J[(size_t)perm[t] * b + i] * sigma[t];
    }
  }
}
__global__ void k_svd_outputs(const double* __restrict__ X, const double* __restrict__ J, int b, int c, int r,
                              const int* __restrict__ perm, const double* __restrict__ sigma, double* Vt,
                              double* W) { k_svd_outputs_body(X, J, b, c, r, perm, sigma, Vt, W); }

int launch_svd_outputs(vp_ctx* ctx, const double* X, const double* J, int b, int c, int r, const int* perm,
                       const double* sigma, double* Vt, double* W) {
  const size_t total = (size_t)r * c + (size_t)b * r;
  const int blocks = (int)std::min<size_t>((total + 255) / 256, (size_t)ctx->num_sms * 8);
  ctx->launches++;
  k_svd_outputs<<<std::max(1, blocks), 256, 0, ctx->stream>>>(X, J, b, c, r, perm, sigma, Vt, W);
  return check_launch(ctx, "svd_outputs");
}

// ------------------------------------------------------ SVD preconditioning
// Static pivoting for the Jacobi SVD: order the columns (tall) or rows (wide)
// of M by decreasing norm, so that the triangular factor of the reordered
// matrix is graded and one-sided Jacobi on it converges in fewer sweeps.
__device__ __forceinline__ void k_norm_order_body(const double* __restrict__ M, int m, int c, int by_cols, int* __restrict__ piv) {
  extern __shared__ double nrm[];
  const int q = by_cols ? c : m, len = by_cols ? m : c;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j < q; j += nw) {
    double a = 0.0;
    for (int i = lane; i < len; i += 32) {
      const double u = by_cols ? M[(size_t)i * c + j] : M[(size_t)j * c + i];
      a = fma(u, u, a);
    }
    a = warp_sum(a);
    if (lane == 0) nrm[j] = a;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < q; j += blockDim.x) {
    const double v = nrm[j];
    int pos = 0;
    for (int k = 0; k < q; ++k) pos += sorts_before(nrm[k], k, v, j);
    piv[pos] = j;
  }
}
__global__ void k_norm_order(const double* __restrict__ M, int m, int c, int by_cols, int* __restrict__ piv) { k_norm_order_body(M, m, c, by_cols, piv); }

int launch_norm_order(vp_ctx* ctx, const double* M, int m, int c, int by_cols, int* piv) {
  const int q = by_cols ? c : m;
  const size_t smem = (size_t)q * sizeof(double);
  if (smem > 200 * 1024) return fail(ctx, VP_ECAPACITY, "norm_order: too many columns");
  if (smem > 48 * 1024) {
    static AttrOnce nattr;  // the largest size once, never lowered under another thread's launch
    VP_TRY(nattr.ensure(ctx, (const void*)k_norm_order, 200 * 1024, false));
  }
  ctx->launches++;
  k_norm_order<<<1, 512, smem, ctx->stream>>>(M, m, c, by_cols, piv);
  return check_launch(ctx, "norm_order");
}

// Column-major copy of the reordered matrix: tall, A = M[:, piv] (m x c);
// wide, A = (M[piv, :])^T (c x m).
__device__ __forceinline__ void k_gather_cm_body(const double* __restrict__ M, int m, int c, const int* __restrict__ piv, int tall,
                            double* __restrict__ out) {
  const size_t total = (size_t)m * c;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    if (tall) {
      const size_t j = e / m, i = e % m;  // out[j*m + i] = M[i][piv[j]]
      out[e] = M[i * c + piv[j]];
    } else {
      const size_t j = e / c, i = e % c;  // out[j*c + i] = M[piv[j]][i]
      out[e] = M[(size_t)piv[j] * c + i];
    }
  }
}
__global__ void k_gather_cm(const double* __restrict__ M, int m, int c, const int* __restrict__ piv, int tall,
                            double* __restrict__ out) { k_gather_cm_body(M, m, c, piv, tall, out); }

int launch_gather_cm(vp_ctx* ctx, const double* M, int m, int c, const int* piv, int tall, double* out) {
  const size_t total = (size_t)m * c;
  const int blocks = (int)std::max<size_t>(1, std::min<size_t>((total + 255) / 256, (size_t)ctx->num_sms * 16));
  ctx->launches++;
  k_gather_cm<<<blocks, 256, 0, ctx->stream>>>(M, m, c, piv, tall, out);
  return check_launch(ctx, "gather_cm");
}

// L = R^T, row-major, from a factored column-major q x q matrix whose upper
// triangle holds R (the reflectors below are dropped).
__device__ __forceinline__ void k_lower_from_upper_body(const double* __restrict__ Rcm, int q, double* __restrict__ L) {
  const size_t total = (size_t)q * q;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = e / q, j = e % q;
    L[e] = (j <= i) ? Rcm[e] : 0.0;
  }
}
__global__ void k_lower_from_upper(const double* __restrict__ Rcm, int q, double* __restrict__ L) { k_lower_from_upper_body(Rcm, q, L); }

int launch_lower_from_upper(vp_ctx* ctx, const double* Rcm, int q, double* L) {
  const size_t total = (size_t)q * q;
  const int blocks = (int)std::max<size_t>(1, std::min<size_t>((total + 255) / 256, (size_t)ctx->num_sms * 8));
  ctx->launches++;
  k_lower_from_upper<<<blocks, 256, 0, ctx->stream>>>(Rcm, q, L);
  return check_launch(ctx, "lower_from_upper");
}

// Undo the static pivoting: cols = 1: out[t][piv[j]] = Y[t][j] (rows x q);
// cols = 0: out[piv[j]][t] = Y[j][t] (q x rows_len).
__device__ __forceinline__ void k_scatter_body(const double* __restrict__ Y, int rows, int cols_n, const int* __restrict__ piv, int cols,
                          double* __restrict__ out) {
  const size_t total = (size_t)rows * cols_n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t a = e / cols_n, b = e % cols_n;
    if (cols)
      out[a * cols_n + piv[b]] = Y[e];
    else
      out[(size_t)piv[a] * cols_n + b] = Y[e];
  }
}
__global__ void k_scatter(const double* __restrict__ Y, int rows, int cols_n, const int* __restrict__ piv, int cols,
                          double* __restrict__ out) { k_scatter_body(Y, rows, cols_n, piv, cols, out); }

int launch_scatter(vp_ctx* ctx, const double* Y, int rows, int cols_n, const int* piv, int cols, double* out) {
  const size_t total = (size_t)rows * cols_n;
  const int blocks = (int)std::max<size_t>(1, std::min<size_t>((total + 255) / 256, (size_t)ctx->num_sms * 8));
  ctx->launches++;
  k_scatter<<<blocks, 256, 0, ctx->stream>>>(Y, rows, cols_n, piv, cols, out);
  return check_launch(ctx, "scatter");
}

// Wide-case outputs: Urows (r x b) = J[perm[t]] (rows of the accumulated
// rotation), Wv (b x r) = X[perm[t]][i] (= V diag(s) of the factor).
__device__ __forceinline__ void k_svd_outputs_wide_body(const double* __restrict__ X, const double* __restrict__ J, int b, int r,
                                   const int* __restrict__ perm, double* Urows, double* Wv) {
  const size_t nu = (size_t)r * b;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < 2 * nu; e += (size_t)gridDim.x * blockDim.x) {
    if (e < nu) {
      const int t = (int)(e / b), q = (int)(e % b);
      Urows[e] = J[(size_t)perm[t] * b + q];
    } else {
      const size_t f = e - nu;
      const int i = (int)(f / r), t = (int)(f % r);
      Wv[f] = X[(size_t)perm[t] * b + i];
    }
  }
}
__global__ void k_svd_outputs_wide(const double* __restrict__ X, const double* __restrict__ J, int b, int r,
                                   const int* __restrict__ perm, double* Urows, double* Wv) { k_svd_outputs_wide_body(X, J, b, r, perm, Urows, Wv); }

int launch_svd_outputs_wide(vp_ctx* ctx, const double* X, const double* J, int b, int r, const int* perm,
                            double* Urows, double* Wv) {
  const size_t total = 2 * (size_t)r * b;
  const int blocks = (int)std::max<size_t>(1, std::min<size_t>((total + 255) / 256, (size_t)ctx->num_sms * 8));
  ctx->launches++;
  k_svd_outputs_wide<<<blocks, 256, 0, ctx->stream>>>(X, J, b, r, perm, Urows, Wv);
  return check_launch(ctx, "svd_outputs_wide");
}

// ====================================================== batched launches
// Each kernel below runs the body of its single-problem counterpart for the
// problem the grid's batch coordinate selects (y for one-dimensional grids,
// z for tiled ones), with that problem's own launch geometry.

void release_scratch(vp_ctx* ctx, BScratch& s) {
  for (DevBuf* b : {&s.wq, &s.wr, &s.qrv, &s.qrc}) release(ctx, *b);
  for (int i = 0; i < kScratchSlots; ++i) {
    release(ctx, s.fq[i]);
    release(ctx, s.qscr[i]);
    release(ctx, s.split[i]);
  }
}

namespace {
// Slot of a job's scratch within one launcher call: the n-th job naming the
// same BScratch takes slot n.
struct SlotCounter {
  std::vector<std::pair<const BScratch*, int>> seen;
  int next(vp_ctx* ctx, const BScratch* s, int* slot) {
    for (auto& e : seen)
      if (e.first == s) {
        if (e.second >= kScratchSlots) return fail(ctx, VP_ECAPACITY, "batched launch: too many jobs on one scratch");
        *slot = e.second++;
        return VP_OK;
      }
    seen.push_back({s, 1});
    *slot = 0;
    return VP_OK;
  }
};
}  // namespace

namespace {

size_t grid_stride_blocks(const vp_ctx* ctx, size_t total, size_t cap_per_sm) {
  return std::max<size_t>(1, std::min<size_t>((total + 255) / 256, (size_t)ctx->num_sms * cap_per_sm));
}

// kern<<<(gx, nb), threads, smem>>>(pack) for every pack of the problems;
// gx(problem) gives the x extent a problem's own launch would use.
template <class A, class GX>
int run_packs(vp_ctx* ctx, cudaStream_t st, const std::vector<A>& v, void (*kern)(const Pack<A>), int threads,
              size_t smem, GX gx, const char* what) {
  for (size_t i0 = 0; i0 < v.size(); i0 += kMaxBatch) {
    const int nb = (int)std::min<size_t>(kMaxBatch, v.size() - i0);
    Pack<A> pk{};
    int gxm = 1;
    for (int i = 0; i < nb; ++i) {
      pk.a[i] = v[i0 + i];
      gxm = std::max(gxm, (int)gx(v[i0 + i]));
    }
    ctx->launches++;
    kern<<<dim3(gxm, nb), threads, smem, st>>>(pk);
    VP_TRY(check_launch(ctx, what));
  }
  return VP_OK;
}

// The same for cluster kernels: grid (cs, nb), clusters of cs CTAs along x.
template <class A>
int run_cluster_packs(vp_ctx* ctx, cudaStream_t st, const std::vector<A>& v, void (*kern)(const Pack<A>), int cs,
                      int threads, size_t smem) {
  for (size_t i0 = 0; i0 < v.size(); i0 += kMaxBatch) {
    const int nb = (int)std::min<size_t>(kMaxBatch, v.size() - i0);
    Pack<A> pk{};
    for (int i = 0; i < nb; ++i) pk.a[i] = v[i0 + i];
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    cfg.gridDim = dim3(cs, nb);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    ctx->launches++;
    VP_CUDA(ctx, cudaLaunchKernelEx(&cfg, kern, pk));
  }
  return VP_OK;
}

}  // namespace

__global__ void kb_to_colmajor(const __grid_constant__ Pack<BColMajor> pk) {
  const BColMajor& a = pk.a[blockIdx.z];
  __shared__ double tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  if (bx >= a.n || by >= a.m) return;  // the whole block is outside this problem
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int r = by + y, c = bx + threadIdx.x;
    if (r < a.m && c < a.n) tile[y][threadIdx.x] = a.A[(size_t)r * a.n + c];
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int c = bx + y, r = by + threadIdx.x;
    if (r < a.m && c < a.n) a.out[(size_t)c * a.m + r] = tile[threadIdx.x][y];
  }
}

int blaunch_to_colmajor(vp_ctx* ctx, cudaStream_t st, const std::vector<BColMajor>& v) {
  for (size_t i0 = 0; i0 < v.size(); i0 += kMaxBatch) {
    const int nb = (int)std::min<size_t>(kMaxBatch, v.size() - i0);
    Pack<BColMajor> pk{};
    int gx = 1, gy = 1;
    for (int i = 0; i < nb; ++i) {
      pk.a[i] = v[i0 + i];
      gx = std::max(gx, (v[i0 + i].n + 31) / 32);
      gy = std::max(gy, (v[i0 + i].m + 31) / 32);
    }
    ctx->launches++;
    kb_to_colmajor<<<dim3(gx, gy, nb), dim3(32, 8), 0, st>>>(pk);
    VP_TRY(check_launch(ctx, "b_to_colmajor"));
  }
  return VP_OK;
}

// --------------------------------------------------------------- QR
struct QRArgs {
  double* A;
  int m, n;
  double* tau;
};
__global__ void __launch_bounds__(kThreads) kb_qr_factor_cdw(const __grid_constant__ Pack<QRArgs> pk) {
  const QRArgs& a = pk.a[blockIdx.y];
  k_qr_factor_cdw_body(a.A, a.m, a.n, a.tau);
}
template <int NT, int CW>
__global__ void __launch_bounds__(NT) kb_qr_factor_cl(const __grid_constant__ Pack<QRArgs> pk) {
  const QRArgs& a = pk.a[blockIdx.y];
  k_qr_factor_cl_body<NT, CW>(a.A, a.m, a.n, a.tau);
}

// Several grid factors in one cooperative launch: problem i owns blocks
// first .. first + nblocks - 1 and runs k_qr_factor_dw's body on them as if
// they were its whole grid (the result does not depend on the block count).
struct QRGridArgs {
  double* A;
  int m, n;
  double* tau;
  dw* V;
  dw* T;
  dw* gcols;
  int* gexp;
  DevStatus* st;
  int first, nblocks;
};
__global__ void __launch_bounds__(kThreads) kb_qr_factor_dw(const __grid_constant__ Pack<QRGridArgs> pk, int count) {
  int i = 0;
  while (i + 1 < count && (int)blockIdx.x >= pk.a[i + 1].first) ++i;
  const QRGridArgs& a = pk.a[i];
  qr_factor_dw_body(a.A, a.m, a.n, a.tau, a.V, a.T, a.gcols, a.gexp, a.st, a.nblocks, blockIdx.x - a.first);
}

// The grid factors of a batch: each launch takes up to kMaxBatch problems
// that each get at least two blocks, one block per SM in all.
static int grid_qr_batch(vp_ctx* ctx, cudaStream_t st, const std::vector<const BQR*>& v) {
  static AttrOnce qattr;
  VP_TRY(qattr.ensure(ctx, (const void*)kb_qr_factor_dw, 200 * 1024, false));
  const int per_launch = std::min(kMaxBatch, std::max(1, ctx->num_sms / 2));
  for (size_t i0 = 0; i0 < v.size(); i0 += per_launch) {
    const int cnt = (int)std::min<size_t>(per_launch, v.size() - i0);
    const int share = std::max(2, ctx->num_sms / cnt);
    Pack<QRGridArgs> pk{};
    int total = 0;
    size_t smem = 0;
    for (int c = 0; c < cnt; ++c) {
      const BQR& q = *v[i0 + c];
      const int p = std::min(q.m, q.n);
      const int blocks = std::max(2, std::min(share, q.n / 2));
      const int nmax = (q.n + blocks - 1) / blocks;
      const size_t need = (size_t)nmax * q.m * sizeof(dw) + (size_t)nmax * sizeof(int);
      VP_TRY(reserve(ctx, q.s->qrv, (size_t)q.m * p + p + 8));
      QRGridArgs& a = pk.a[c];
      a = {q.A, q.m, q.n, q.tau, reinterpret_cast<dw*>(q.s->qrv.p), nullptr, nullptr, nullptr, q.s->st, total, blocks};
      a.T = a.V + (size_t)q.m * p;
      if (need > 200 * 1024) {  // columns in global scratch
        VP_TRY(reserve(ctx, q.s->qrc, (size_t)q.m * q.n + q.n / 2 + 8));
        a.gcols = reinterpret_cast<dw*>(q.s->qrc.p);
        a.gexp = reinterpret_cast<int*>(a.gcols + (size_t)q.m * q.n);
      } else {
        smem = std::max(smem, need);
      }
      total += blocks;
    }
    int count = cnt;
    void* args[] = {&pk, &count};
    VP_TRY(coop_launch(ctx, st, (const void*)kb_qr_factor_dw, total, kThreads, args, smem, "b_qr_factor_dw"));
  }
  return VP_OK;
}

int blaunch_qr_factor(vp_ctx* ctx, cudaStream_t st, const std::vector<BQR>& v) {
  std::vector<BQR> wide;
  std::vector<const BQR*> grid;
  std::vector<QRArgs> cdw[17], cl[17];
  size_t cdw_smem[17] = {}, cl_smem[17] = {};
  // More than four cluster factors in one call: 8-CTA clusters where they fit,
  // so that twice as many problems run side by side (the result does not
  // depend on the CTA count).
  int ncl = 0;
  for (const BQR& q : v) ncl += qr_plan(ctx, q.m, q.n).kind == QR_CL;
  for (const BQR& q : v) {
    QRPlan pl = qr_plan(ctx, q.m, q.n);
    if (pl.kind == QR_CL && ncl > 4 && pl.cs > 8 && qr_cl_smem(q.m, q.n, 8) <= 200 * 1024) pl.cs = 8;
    switch (pl.kind) {
      case QR_NONE:
        break;
      case QR_WIDE:
        wide.push_back(q);
        break;
      case QR_CDW:
        cdw[pl.cs].push_back({q.A, q.m, q.n, q.tau});
        cdw_smem[pl.cs] = std::max(cdw_smem[pl.cs], qr_cdw_smem(q.m, q.n, pl.cs));
        break;
      case QR_CL:
        cl[pl.cs].push_back({q.A, q.m, q.n, q.tau});
        cl_smem[pl.cs] = std::max(cl_smem[pl.cs], qr_cl_smem(q.m, q.n, pl.cs));
        break;
      default:
        if (!q.s || !q.s->st) return fail(ctx, VP_EINVAL, "batched QR: no status words for a grid factor");
        if (q.n / 2 >= 2)
          grid.push_back(&q);
        else  // a single block: the barrier kernel of the single path
          VP_TRY(qr_factor_grid(ctx, st, q.s->st, q.s->qrv, q.s->qrc, q.A, q.m, q.n, q.tau, q.vbuf));
    }
  }
  for (int cs = 1; cs <= 16; ++cs) {
    if (!cdw[cs].empty()) {
      static AttrOnce a;
      VP_TRY(a.ensure(ctx, (const void*)kb_qr_factor_cdw, 200 * 1024, true));
      VP_TRY(run_cluster_packs(ctx, st, cdw[cs], kb_qr_factor_cdw, cs, kThreads,
                               std::max<size_t>(cdw_smem[cs], 116 * 1024)));
    }
    if (!cl[cs].empty()) {
      static AttrOnce a;
      VP_TRY(a.ensure(ctx, (const void*)kb_qr_factor_cl<512, 4>, 200 * 1024, true));
      VP_TRY(run_cluster_packs(ctx, st, cl[cs], kb_qr_factor_cl<512, 4>, cs, 512,
                               std::max<size_t>(cl_smem[cs], 116 * 1024)));
    }
  }
  if (!grid.empty()) VP_TRY(grid_qr_batch(ctx, st, grid));
  if (!wide.empty()) {  // the square block, its Q, R2^T = A2^T Q in FP64, copied back (see qr_plan)
    std::vector<BQR> sq;
    std::vector<BFormQ> fq;
    std::vector<BGemm> gm;
    std::vector<BCopy> cp;
    for (const BQR& q : wide) {
      const int m = q.m;
      const size_t rest = (size_t)(q.n - m) * m;
      VP_TRY(reserve(ctx, q.s->wq, (size_t)m * m));
      VP_TRY(reserve(ctx, q.s->wr, rest));
      sq.push_back({q.A, m, m, q.tau, q.vbuf, q.s});
      fq.push_back({q.A, m, m, q.tau, q.s->wq.p, q.s});
      gm.push_back({BG_AB, 0, q.n - m, m, m, 1.0, q.A + (size_t)m * m, m, q.s->wq.p, m, q.s->wr.p, m, q.s});
      cp.push_back({q.s->wr.p, q.A + (size_t)m * m, rest});
    }
    VP_TRY(blaunch_qr_factor(ctx, st, sq));
    VP_TRY(blaunch_qr_formq(ctx, st, fq));
    VP_TRY(blaunch_gemm(ctx, st, gm));
    VP_TRY(blaunch_copy(ctx, st, cp));
  }
  return VP_OK;
}

struct R2DwArgs {
  const double* A;
  int m, p;
  const double* tau;
  dw* V;
  dw* T;
};
__global__ void kb_reflectors_to_dw(const __grid_constant__ Pack<R2DwArgs> pk) {
  const R2DwArgs& a = pk.a[blockIdx.y];
  k_reflectors_to_dw_body(a.A, a.m, a.p, a.tau, a.V, a.T);
}
struct FormQArgs {
  const dw* V;
  int m, p;
  const dw* T;
  dw* scratch;
  double* Q;
};
template <int R>
__global__ void kb_qr_formq_reg(const __grid_constant__ Pack<FormQArgs> pk) {
  const FormQArgs& a = pk.a[blockIdx.y];
  k_qr_formq_reg_body<R>(a.V, a.m, a.p, a.T, a.Q);
}
__global__ void kb_qr_formq_dw(const __grid_constant__ Pack<FormQArgs> pk) {
  const FormQArgs& a = pk.a[blockIdx.y];
  k_qr_formq_dw_body(a.V, a.m, a.p, a.T, a.scratch, a.Q);
}

int blaunch_qr_formq(vp_ctx* ctx, cudaStream_t st, const std::vector<BFormQ>& v) {
  std::vector<R2DwArgs> conv;
  std::vector<FormQArgs> reg[5], gl;
  SlotCounter slots;
  for (const BFormQ& f : v) {
    const int p = std::min(f.m, f.n);
    if (p <= 0) continue;
    int sl = 0;
    VP_TRY(slots.next(ctx, f.s, &sl));
    VP_TRY(reserve(ctx, f.s->fq[sl], (size_t)f.m * p + p + 8));
    dw* V = reinterpret_cast<dw*>(f.s->fq[sl].p);
    dw* T = V + (size_t)f.m * p;
    conv.push_back({f.A, f.m, p, f.tau, V, T});
    FormQArgs a{V, f.m, p, T, nullptr, f.Q};
    if (f.m <= 64) reg[1].push_back(a);
    else if (f.m <= 128) reg[2].push_back(a);
    else if (f.m <= 256) reg[3].push_back(a);
    else if (f.m <= 512) reg[4].push_back(a);
    else {
      VP_TRY(reserve(ctx, f.s->qscr[sl], (size_t)f.m * p));
      a.scratch = reinterpret_cast<dw*>(f.s->qscr[sl].p);
      gl.push_back(a);
    }
  }
  VP_TRY(run_packs(ctx, st, conv, kb_reflectors_to_dw, 256, 0,
                   [&](const R2DwArgs& a) { return grid_stride_blocks(ctx, (size_t)a.m * a.p, 8); }, "b_refl_to_dw"));
  auto blocks4 = [](const FormQArgs& a) { return (a.p + 3) / 4; };
  VP_TRY(run_packs(ctx, st, reg[1], kb_qr_formq_reg<2>, 128, 0, blocks4, "b_formq"));
  VP_TRY(run_packs(ctx, st, reg[2], kb_qr_formq_reg<4>, 128, 0, blocks4, "b_formq"));
  VP_TRY(run_packs(ctx, st, reg[3], kb_qr_formq_reg<8>, 128, 0, blocks4, "b_formq"));
  VP_TRY(run_packs(ctx, st, reg[4], kb_qr_formq_reg<16>, 128, 0, blocks4, "b_formq"));
  return run_packs(ctx, st, gl, kb_qr_formq_dw, 256, 0, [](const FormQArgs& a) { return (a.p + 7) / 8; },
                   "b_formq_dw");
}

struct GetRArgs {
  const double* A;
  int m, n, p;
  double* R;
};
__global__ void kb_qr_getr(const __grid_constant__ Pack<GetRArgs> pk) {
  const GetRArgs& a = pk.a[blockIdx.y];
  k_qr_getr_body(a.A, a.m, a.n, a.p, a.R);
}
int blaunch_qr_getr(vp_ctx* ctx, cudaStream_t st, const std::vector<BGetR>& v) {
  std::vector<GetRArgs> g;
  for (const BGetR& r : v) {
    const int p = std::min(r.m, r.n);
    if ((size_t)p * r.n > 0) g.push_back({r.A, r.m, r.n, p, r.R});
  }
  return run_packs(ctx, st, g, kb_qr_getr, 256, 0,
                   [&](const GetRArgs& a) { return grid_stride_blocks(ctx, (size_t)a.p * a.n, 16); }, "b_getr");
}

// --------------------------------------------------------------- GEMM
template <class ALoad, class BLoad>
struct GemmJob {
  int M, N, K, kslice, slices;
  double alpha;
  ALoad a;
  BLoad b;
  double* C;
  int ldc;
  size_t stride;
};
template <class ALoad, class BLoad, class T, int TILE>
__global__ void __launch_bounds__(256) kb_gemm(const __grid_constant__ Pack<GemmJob<ALoad, BLoad>> pk, int zs) {
  const GemmJob<ALoad, BLoad>& j = pk.a[blockIdx.z / zs];
  const int slice = blockIdx.z % zs;
  if (slice >= j.slices || (int)blockIdx.x * TILE >= j.M || (int)blockIdx.y * TILE >= j.N) return;
  gemm_body<ALoad, BLoad, T, TILE>(j.M, j.N, j.K, j.alpha, j.a, j.b, j.C, j.ldc, j.kslice, j.stride, blockIdx.x,
                                   blockIdx.y, slice);
}
struct SumArgs {
  const double* P;
  int M, N, slices;
  size_t stride;
  double* C;
  int ldc;
};
__global__ void kb_sum_slices(const __grid_constant__ Pack<SumArgs> pk) {
  const SumArgs& a = pk.a[blockIdx.y];
  k_sum_slices_body(a.P, a.M, a.N, a.slices, a.stride, a.C, a.ldc);
}

namespace {
template <class ALoad, class BLoad, class T, int TILE>
int gemm_group(vp_ctx* ctx, cudaStream_t st, const std::vector<GemmJob<ALoad, BLoad>>& jobs) {
  for (size_t i0 = 0; i0 < jobs.size(); i0 += kMaxBatch) {
    const int nb = (int)std::min<size_t>(kMaxBatch, jobs.size() - i0);
    Pack<GemmJob<ALoad, BLoad>> pk{};
    int gx = 1, gy = 1, zs = 1;
    for (int i = 0; i < nb; ++i) {
      const auto& j = jobs[i0 + i];
      pk.a[i] = j;
      gx = std::max(gx, (j.M + TILE - 1) / TILE);
      gy = std::max(gy, (j.N + TILE - 1) / TILE);
      zs = std::max(zs, j.slices);
    }
    if (gy > 65535) return fail(ctx, VP_ECAPACITY, "gemm: N too large");
    ctx->launches++;
    kb_gemm<ALoad, BLoad, T, TILE><<<dim3(gx, gy, nb * zs), 256, 0, st>>>(pk, zs);
    VP_TRY(check_launch(ctx, "b_gemm"));
  }
  return VP_OK;
}
}  // namespace

int blaunch_gemm(vp_ctx* ctx, cudaStream_t st, const std::vector<BGemm>& v) {
  // [FP32 contraction][tile 64 / 32]
  std::vector<GemmJob<ARowMajor, BRowMajor>> ab[2][2];
  std::vector<GemmJob<ARowMajor, BTransposed>> abt[2][2];
  std::vector<GemmJob<AUpperColMajor, BRowMajor>> rb[2][2];
  std::vector<SumArgs> sums;
  SlotCounter slots;
  for (const BGemm& g : v) {
    if (g.M <= 0 || g.N <= 0) continue;
    const GemmPlan pl = gemm_plan(ctx, g.M, g.N, g.K);
    const int slices = pl.slices, kslice = pl.kslice, ti = pl.tile == 64 ? 0 : 1;
    double* C = g.C;
    int ldc = g.ldc;
    size_t stride = 0;
    if (slices > 1) {
      int sl = 0;
      VP_TRY(slots.next(ctx, g.s, &sl));
      stride = (size_t)g.M * g.N;
      VP_TRY(reserve(ctx, g.s->split[sl], stride * slices));
      C = g.s->split[sl].p;
      ldc = g.N;
      sums.push_back({g.s->split[sl].p, g.M, g.N, slices, stride, g.C, g.ldc});
    }
    const int t = g.fp32 ? 1 : 0;
    if (g.kind == BG_AB)
      ab[t][ti].push_back({g.M, g.N, g.K, kslice, slices, g.alpha, ARowMajor{g.A, g.lda}, BRowMajor{g.B, g.ldb}, C, ldc,
                       stride});
    else if (g.kind == BG_ABT)
      abt[t][ti].push_back({g.M, g.N, g.K, kslice, slices, g.alpha, ARowMajor{g.A, g.lda}, BTransposed{g.B, g.ldb}, C,
                        ldc, stride});
    else
      rb[t][ti].push_back({g.M, g.N, g.K, kslice, slices, g.alpha, AUpperColMajor{g.A, g.lda}, BRowMajor{g.B, g.ldb}, C,
                       ldc, stride});
  }
  VP_TRY((gemm_group<ARowMajor, BRowMajor, double, 64>(ctx, st, ab[0][0])));
  VP_TRY((gemm_group<ARowMajor, BRowMajor, double, 32>(ctx, st, ab[0][1])));
  VP_TRY((gemm_group<ARowMajor, BRowMajor, float, 64>(ctx, st, ab[1][0])));
  VP_TRY((gemm_group<ARowMajor, BRowMajor, float, 32>(ctx, st, ab[1][1])));
  VP_TRY((gemm_group<ARowMajor, BTransposed, double, 64>(ctx, st, abt[0][0])));
  VP_TRY((gemm_group<ARowMajor, BTransposed, double, 32>(ctx, st, abt[0][1])));
  VP_TRY((gemm_group<ARowMajor, BTransposed, float, 64>(ctx, st, abt[1][0])));
  VP_TRY((gemm_group<ARowMajor, BTransposed, float, 32>(ctx, st, abt[1][1])));
  VP_TRY((gemm_group<AUpperColMajor, BRowMajor, double, 64>(ctx, st, rb[0][0])));
  VP_TRY((gemm_group<AUpperColMajor, BRowMajor, double, 32>(ctx, st, rb[0][1])));
  VP_TRY((gemm_group<AUpperColMajor, BRowMajor, float, 64>(ctx, st, rb[1][0])));
  VP_TRY((gemm_group<AUpperColMajor, BRowMajor, float, 32>(ctx, st, rb[1][1])));
  return run_packs(ctx, st, sums, kb_sum_slices, 256, 0,
                   [&](const SumArgs& a) { return grid_stride_blocks(ctx, a.stride, 8); }, "b_sum_slices");
}

// --------------------------------------------------------------- SVD site helpers
__global__ void kb_norm_order(const __grid_constant__ Pack<BNormOrder> pk) {
  const BNormOrder& a = pk.a[blockIdx.y];
  k_norm_order_body(a.M, a.m, a.c, a.by_cols, a.piv);
}
int blaunch_norm_order(vp_ctx* ctx, cudaStream_t st, const std::vector<BNormOrder>& v) {
  size_t smem = 0;
  for (const BNormOrder& a : v) smem = std::max(smem, (size_t)(a.by_cols ? a.c : a.m) * sizeof(double));
  if (smem > 200 * 1024) return fail(ctx, VP_ECAPACITY, "norm_order: too many columns");
  static AttrOnce at;
  VP_TRY(at.ensure(ctx, (const void*)kb_norm_order, 200 * 1024, false));
  return run_packs(ctx, st, v, kb_norm_order, 512, smem, [](const BNormOrder&) { return 1; }, "b_norm_order");
}
__global__ void kb_gather_cm(const __grid_constant__ Pack<BGather> pk) {
  const BGather& a = pk.a[blockIdx.y];
  k_gather_cm_body(a.M, a.m, a.c, a.piv, a.tall, a.out);
}
int blaunch_gather_cm(vp_ctx* ctx, cudaStream_t st, const std::vector<BGather>& v) {
  return run_packs(ctx, st, v, kb_gather_cm, 256, 0,
                   [&](const BGather& a) { return grid_stride_blocks(ctx, (size_t)a.m * a.c, 16); }, "b_gather_cm");
}
__global__ void kb_lower_from_upper(const __grid_constant__ Pack<BLowerUpper> pk) {
  const BLowerUpper& a = pk.a[blockIdx.y];
  k_lower_from_upper_body(a.R, a.q, a.L);
}
int blaunch_lower_from_upper(vp_ctx* ctx, cudaStream_t st, const std::vector<BLowerUpper>& v) {
  return run_packs(ctx, st, v, kb_lower_from_upper, 256, 0,
                   [&](const BLowerUpper& a) { return grid_stride_blocks(ctx, (size_t)a.q * a.q, 8); },
                   "b_lower_from_upper");
}

struct JacArgs {
  double* X;
  int b, c;
  double* J;
  float eps;
  int max_sweeps, nb;
  DevStatus* st;
};
__global__ void __launch_bounds__(kThreads) kb_jacobi_dw(const __grid_constant__ Pack<JacArgs> pk) {
  const JacArgs& a = pk.a[blockIdx.y];
  k_jacobi_dw_body(a.X, a.b, a.c, a.J, a.eps, a.max_sweeps, a.nb, a.st);
}
int blaunch_jacobi(vp_ctx* ctx, cudaStream_t st, const std::vector<BJacobi>& v) {
  const int CS = ctx->cluster_size;
  std::vector<JacArgs> grp[17];
  size_t smem[17] = {};
  for (const BJacobi& j : v) {
    if (j.b <= 1) continue;  // nothing to rotate (as in the single launch)
    const JacBlockCfg bc = jac_block_cfg(j.b, j.c, j.J != nullptr, std::max(1, CS));
    if (jac_dw_smem(bc) <= 200 * 1024) {
      // the thresholds of launch_jacobi_rows
      grp[bc.CS].push_back({j.X, j.b, j.c, j.J, (float)(4e-13 * std::sqrt((double)j.c)), 60, bc.nb, j.st});
      smem[bc.CS] = std::max(smem[bc.CS], jac_dw_smem(bc));
    } else {
      VP_CUDA(ctx, cudaMemsetAsync(j.st->rot, 0, sizeof(j.st->rot), st));
      VP_TRY(jacobi_rows_on(ctx, st, j.st, j.X, j.b, j.c, j.J, true));
    }
  }
  for (int cs = 1; cs <= 16; ++cs)
    if (!grp[cs].empty()) {
      static AttrOnce a;
      VP_TRY(a.ensure(ctx, (const void*)kb_jacobi_dw, 200 * 1024, true));
      VP_TRY(run_cluster_packs(ctx, st, grp[cs], kb_jacobi_dw, cs, kThreads, std::max<size_t>(smem[cs], 120 * 1024)));
    }
  return VP_OK;
}

__global__ void kb_select(const __grid_constant__ Pack<BSelect> pk) {
  const BSelect& a = pk.a[blockIdx.y];
  k_select_body(a.X, a.b, a.c, a.chi, a.tol, a.perm, a.sigma, a.d_rank, a.d_err, a.st);
}
int blaunch_select(vp_ctx* ctx, cudaStream_t st, const std::vector<BSelect>& v) {
  size_t smem = 0;
  for (const BSelect& a : v) smem = std::max(smem, (size_t)(2 * a.b + 1) * sizeof(double));
  if (smem > 200 * 1024) return fail(ctx, VP_ECAPACITY, "select: bond too large");
  static AttrOnce at;
  VP_TRY(at.ensure(ctx, (const void*)kb_select, 200 * 1024, false));
  return run_packs(ctx, st, v, kb_select, 512, smem, [](const BSelect&) { return 1; }, "b_select");
}
__global__ void kb_svd_outputs(const __grid_constant__ Pack<BSvdOut> pk) {
  const BSvdOut& a = pk.a[blockIdx.y];
  k_svd_outputs_body(a.X, a.J, a.b, a.c, a.r, a.perm, a.sigma, a.Vt, a.W);
}
int blaunch_svd_outputs(vp_ctx* ctx, cudaStream_t st, const std::vector<BSvdOut>& v) {
  return run_packs(ctx, st, v, kb_svd_outputs, 256, 0,
                   [&](const BSvdOut& a) {
                     return grid_stride_blocks(ctx, (size_t)a.r * a.c + (size_t)a.b * a.r, 8);
                   },
                   "b_svd_outputs");
}
__global__ void kb_svd_outputs_wide(const __grid_constant__ Pack<BSvdOutWide> pk) {
  const BSvdOutWide& a = pk.a[blockIdx.y];
  k_svd_outputs_wide_body(a.X, a.J, a.b, a.r, a.perm, a.U, a.Wv);
}
int blaunch_svd_outputs_wide(vp_ctx* ctx, cudaStream_t st, const std::vector<BSvdOutWide>& v) {
  return run_packs(ctx, st, v, kb_svd_outputs_wide, 256, 0,
                   [&](const BSvdOutWide& a) { return grid_stride_blocks(ctx, 2 * (size_t)a.r * a.b, 8); },
                   "b_svd_outputs_wide");
}
__global__ void kb_scatter(const __grid_constant__ Pack<BScatter> pk) {
  const BScatter& a = pk.a[blockIdx.y];
  k_scatter_body(a.Y, a.rows, a.cols_n, a.piv, a.cols, a.out);
}
int blaunch_scatter(vp_ctx* ctx, cudaStream_t st, const std::vector<BScatter>& v) {
  return run_packs(ctx, st, v, kb_scatter, 256, 0,
                   [&](const BScatter& a) { return grid_stride_blocks(ctx, (size_t)a.rows * a.cols_n, 8); },
                   "b_scatter");
}

}  // namespace vp
