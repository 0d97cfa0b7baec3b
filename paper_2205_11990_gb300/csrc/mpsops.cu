// Memory-bound MPS/MPO kernels: per-site MPO x MPS contraction fused with MPS
// addition (SI "Matrix-vector multiplication", "Addition"), integration over v
// (SI "Integration"), the periodic Poisson solve (main text Eqs. for phi and
// E), the site permutation of the interleaved mapping, and the assembly of
// the Vlasov operator's MPO with the field term (SI "Dot Product").
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"

namespace vp {

static int grid_for(vp_ctx* ctx, size_t total, int per = 256) {
  return (int)std::max<size_t>(1, std::min<size_t>((total + per - 1) / per, (size_t)ctx->num_sms * 16));
}

// out core (ol, 2, orr) = alpha*a (+) beta*(B b), blocks placed as in the
// MPS sum: a occupies the leading block of each bond, (B b) the trailing one
// with bond index (alpha, beta) = a_b * w + b_w; the first site concatenates
// along the right bond only and the last site along the left bond only.
__device__ __forceinline__ void k_site_sum_body(SiteSum s, double* __restrict__ out, int ol, int orr) {
  const size_t total = (size_t)ol * 2 * orr;
  const int offl = (s.a && !s.first) ? s.al : 0;  // start of the (B b) block on the left bond
  const int offr = (s.a && !s.last) ? s.ar : 0;
  const int wl = s.B ? s.wl : 1, wr = s.B ? s.wr : 1;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int l = (int)(e / (2 * orr));
    const int o = (int)((e / orr) & 1);
    const int r = (int)(e % orr);
    double v = 0.0;
    // a block
    if (s.a) {
      const bool inl = s.first ? true : (l < s.al);
      const bool inr = s.last ? true : (r < s.ar);
      if (inl && inr) {
        const int la = s.first ? 0 : l, ra = s.last ? 0 : r;
        v = s.alpha * s.a[((size_t)la * 2 + o) * s.ar + ra];
      }
    }
    // (B b) block
    const bool inl = s.a ? (s.first ? true : l >= offl) : true;
    const bool inr = s.a ? (s.last ? true : r >= offr) : true;
    if (inl && inr) {
      const int lb = s.first ? 0 : l - offl, rb = s.last ? 0 : r - offr;
      const int al = lb / wl, bw = lb % wl, ar = rb / wr, brw = rb % wr;
      double acc;
      if (s.B) {
        const double* Bc = s.B + ((size_t)bw * 4 + o * 2) * wr + brw;  // B[bw][o][i][brw], i stride wr
        const double* bc = s.b + (size_t)al * 2 * s.br + ar;          // b[al][i][ar], i stride br
        acc = Bc[0] * bc[0] + Bc[wr] * bc[s.br];
      } else {
        acc = s.b[((size_t)al * 2 + o) * s.br + ar];
      }
      v += s.beta * acc;
    }
    out[e] = v;
  }
}
__global__ void k_site_sum(SiteSum s, double* __restrict__ out, int ol, int orr) { k_site_sum_body(s, out, ol, orr); }

int launch_site_sum(vp_ctx* ctx, const SiteSum& s, double* out, int ol, int orr) {
  const size_t total = (size_t)ol * 2 * orr;
  ctx->launches++;
  k_site_sum<<<grid_for(ctx, total), 256, 0, ctx->stream>>>(s, out, ol, orr);
  return check_launch(ctx, "site_sum");
}

__device__ __forceinline__ void k_phys_sum_body(const double* __restrict__ core, int rl, int rr, double* __restrict__ T) {
  const size_t total = (size_t)rl * rr;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t l = e / rr, r = e % rr;
    T[e] = core[(l * 2) * rr + r] + core[(l * 2 + 1) * rr + r];
  }
}
__global__ void k_phys_sum(const double* __restrict__ core, int rl, int rr, double* __restrict__ T) { k_phys_sum_body(core, rl, rr, T); }

int launch_phys_sum(vp_ctx* ctx, const double* core, int rl, int rr, double* T) {
  ctx->launches++;
  k_phys_sum<<<grid_for(ctx, (size_t)rl * rr), 256, 0, ctx->stream>>>(core, rl, rr, T);
  return check_launch(ctx, "phys_sum");
}

__device__ __forceinline__ void k_copy_body(const double* __restrict__ src, double* __restrict__ dst, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    dst[e] = src[e];
}
__global__ void k_copy(const double* __restrict__ src, double* __restrict__ dst, size_t n) { k_copy_body(src, dst, n); }

int launch_copy(vp_ctx* ctx, const double* src, double* dst, size_t n) {
  if (n == 0) return VP_OK;
  ctx->launches++;
  k_copy<<<grid_for(ctx, n), 256, 0, ctx->stream>>>(src, dst, n);
  return check_launch(ctx, "copy");
}

__device__ __forceinline__ void k_scale_body(double* x, size_t n, double s) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    x[e] *= s;
}
__global__ void k_scale(double* x, size_t n, double s) { k_scale_body(x, n, s); }

int launch_scale(vp_ctx* ctx, double* x, size_t n, double s) {
  if (n == 0) return VP_OK;
  ctx->launches++;
  k_scale<<<grid_for(ctx, n), 256, 0, ctx->stream>>>(x, n, s);
  return check_launch(ctx, "scale");
}

// A core (a, 2, b) read back to front: out (b, 2, a), out[j][s][i] = in[i][s][j]
// (the same site in a chain taken in the opposite order).
__global__ void k_core_transpose(const double* __restrict__ in, int a, int b, double* __restrict__ out) {
  const size_t total = (size_t)a * 2 * b;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / (2 * (size_t)a)), sb = (int)((e / a) % 2), i = (int)(e % a);
    out[e] = in[((size_t)i * 2 + sb) * b + j];
  }
}

int launch_core_transpose(vp_ctx* ctx, const double* in, int a, int b, double* out) {
  const size_t n = (size_t)a * 2 * b;
  if (n == 0) return VP_OK;
  ctx->launches++;
  k_core_transpose<<<grid_for(ctx, n), 256, 0, ctx->stream>>>(in, a, b, out);
  return check_launch(ctx, "core_transpose");
}

// Row i of a (rows x cols) row-major matrix times s[i] (invert: 1/s[i], and 0
// where s[i] is 0).
__global__ void k_scale_rows(double* x, int rows, int cols, const double* __restrict__ sv, int invert) {
  const size_t total = (size_t)rows * cols;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const double v = sv[e / cols];
    x[e] *= invert ? (v != 0.0 ? 1.0 / v : 0.0) : v;
  }
}

int launch_scale_rows(vp_ctx* ctx, double* x, int rows, int cols, const double* sv, int invert) {
  const size_t n = (size_t)rows * cols;
  if (n == 0) return VP_OK;
  ctx->launches++;
  k_scale_rows<<<grid_for(ctx, n), 256, 0, ctx->stream>>>(x, rows, cols, sv, invert);
  return check_launch(ctx, "scale_rows");
}

// Site-ordered index <-> (ix, iv).  Site order: SEQ = x bits then v bits;
// INTERLEAVED = x0 v0 x1 v1 ... with leftover bits of the longer dimension.
__device__ __forceinline__ size_t bitrev_n(size_t x, int n) { return n > 0 ? __brevll(x) >> (64 - n) : 0; }

__device__ __forceinline__ size_t site_to_grid(size_t s, int nx, int nv, int mapping) {
  if (mapping == VP_SEQ) return s;  // already [ix][iv]
  if (mapping == VP_SEQ_S2 || mapping == VP_SEQ_S3) {
    size_t ix = s >> nv, iv = s & ((size_t(1) << nv) - 1);
    if (mapping == VP_SEQ_S2) ix = bitrev_n(ix, nx);  // x bits fine to coarse
    else iv = bitrev_n(iv, nv);                        // v bits fine to coarse
    return (ix << nv) | iv;
  }
  const int n = nx + nv;
  size_t ix = 0, iv = 0;
  int site = 0;
  const int mx = max(nx, nv);
  for (int b = 0; b < mx; ++b) {
    if (b < nx) {
      ix = (ix << 1) | ((s >> (n - 1 - site)) & 1);
      ++site;
    }
    if (b < nv) {
      iv = (iv << 1) | ((s >> (n - 1 - site)) & 1);
      ++site;
    }
  }
  return (ix << nv) | iv;
}

__device__ __forceinline__ void k_permute_body(const double* __restrict__ f, int nx, int nv, int mapping, double* __restrict__ out,
                          int inverse) {
  const size_t total = (size_t)1 << (nx + nv);
  for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < total; s += (size_t)gridDim.x * blockDim.x) {
    const size_t g = site_to_grid(s, nx, nv, mapping);
    if (inverse)
      out[g] = f[s];
    else
      out[s] = f[g];
  }
}
__global__ void k_permute(const double* __restrict__ f, int nx, int nv, int mapping, double* __restrict__ out,
                          int inverse) { k_permute_body(f, nx, nv, mapping, out, inverse); }

int launch_permute_to_sites(vp_ctx* ctx, const double* f, int nx, int nv, int mapping, double* out,
                            int inverse) {
  const size_t total = (size_t)1 << (nx + nv);
  ctx->launches++;
  k_permute<<<grid_for(ctx, total), 256, 0, ctx->stream>>>(f, nx, nv, mapping, out, inverse);
  return check_launch(ctx, "permute");
}

// Periodic second-order Poisson on one block.  With s_i = dx^2 (rho_i -
// mean) and d_i = phi_{i+1} - phi_i the difference equation reads d_i -
// d_{i-1} = s_i, so d is a prefix sum fixed by sum_i d_i = 0 (periodicity),
// and E_i = -(phi_{i+1} - phi_{i-1}) / (2 dx) = -(d_i + d_{i-1}) / (2 dx).
// we[0] = 1/2 sum E^2 dx, we[1] = sum rho dx.
__device__ __forceinline__ void k_poisson_body(const double* __restrict__ rho, int N, double dx, double* __restrict__ E,
                          double* __restrict__ we) {
  extern __shared__ double sm[];
  double* d = sm;           // N
  double* red = sm + N;     // blockDim/32 + 1
  double* part = red + 33;  // blockDim
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  auto bsum = [&](double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += red[w];
      red[32] = t;
    }
    __syncthreads();
    return red[32];
  };
  double loc = 0.0;
  for (int i = tid; i < N; i += nt) loc += rho[i];
  const double total = bsum(loc);
  const double mean = total / N;
  // contiguous chunk per thread: serial prefix inside, block scan across
  const int chunk = (N + nt - 1) / nt;
  const int lo = min(N, tid * chunk), hi = min(N, lo + chunk);
  double run = 0.0;
  for (int i = lo; i < hi; ++i) {
    // S_i = sum_{j=1}^{i} s_j (S_0 = 0)
    if (i > 0) run += dx * dx * (rho[i] - mean);
    d[i] = run;
  }
  part[tid] = run;
  __syncthreads();
  if (tid == 0) {
    double acc = 0.0;
    for (int t = 0; t < nt; ++t) {
      const double v = part[t];
      part[t] = acc;
      acc += v;
    }
  }
  __syncthreads();
  double sS = 0.0;
  for (int i = lo; i < hi; ++i) {
    d[i] += part[tid];
    sS += d[i];
  }
  const double sumS = bsum(sS);
  const double d0 = -sumS / N;
  for (int i = tid; i < N; i += nt) d[i] += d0;  // d_i = d_0 + S_i
  __syncthreads();
  double e2 = 0.0;
  for (int i = tid; i < N; i += nt) {
    const double dm = d[(i + N - 1) % N];
    const double e = -(d[i] + dm) / (2.0 * dx);
    E[i] = e;
    e2 = fma(e, e, e2);
  }
  const double we_ = bsum(e2);
  if (tid == 0) {
    we[0] = 0.5 * we_ * dx;
    we[1] = total * dx;
  }
}
__global__ void k_poisson(const double* __restrict__ rho, int N, double dx, double* __restrict__ E,
                          double* __restrict__ we) { k_poisson_body(rho, N, dx, E, we); }

int launch_poisson(vp_ctx* ctx, const double* rho, int N, double dx, double* E, double* we_dev) {
  const int nt = 256;
  const size_t smem = (size_t)(N + 33 + nt) * sizeof(double);
  if (smem > 200 * 1024) return fail(ctx, VP_ECAPACITY, "poisson: 2^nx too large");
  if (smem > 48 * 1024) {
    static AttrOnce pattr;  // the largest size once, never lowered under another thread's launch
    VP_TRY(pattr.ensure(ctx, (const void*)k_poisson, 200 * 1024, false));
  }
  ctx->launches++;
  k_poisson<<<1, nt, smem, ctx->stream>>>(rho, N, dx, E, we_dev);
  return check_launch(ctx, "poisson");
}

// Net density of several species, net_i = sum_s w_s rho_s[i], and each
// species' mass sum_i rho_s[i] dx (one block).
__global__ void k_species_net(SpeciesRho sr, int N, double dx, double* __restrict__ net, double* __restrict__ mass) {
  __shared__ double red[32];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < N; i += nt) {
    double a = 0.0;
    for (int s = 0; s < sr.ns; ++s) a = fma(sr.w[s], sr.rho[s][i], a);
    net[i] = a;
  }
  for (int s = 0; s < sr.ns; ++s) {
    double loc = 0.0;
    for (int i = tid; i < N; i += nt) loc += sr.rho[s][i];
    for (int o = 16; o > 0; o >>= 1) loc += __shfl_xor_sync(0xffffffffu, loc, o);
    if (lane == 0) red[warp] = loc;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < nt / 32; ++w) t += red[w];
      mass[s] = t * dx;
    }
    __syncthreads();
  }
}

int launch_species_net(vp_ctx* ctx, const SpeciesRho& sr, int N, double dx, double* net, double* mass) {
  if (sr.ns < 1 || sr.ns > kMaxSpecies) return fail(ctx, VP_EINVAL, "species_net: bad species count");
  ctx->launches++;
  k_species_net<<<1, 256, 0, ctx->stream>>>(sr, N, dx, net, mass);
  return check_launch(ctx, "species_net");
}

// L core = blockdiag(U, T) with T the placed field term diag(E) (x) D_v.
// Bond indices of T flatten (E channel, D_v channel) in that order.
__device__ __forceinline__ void k_assemble_body(const double* __restrict__ U, int ul, int ur, ETermSite e, int first, int last,
                           double* __restrict__ out, int ol, int orr) {
  const size_t total = (size_t)ol * 4 * orr;
  const int tl = first ? 1 : ol - ul;  // T block sizes
  const int tr = last ? 1 : orr - ur;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int l = (int)(q / (4 * orr));
    const int oi = (int)((q / orr) & 3);
    const int o = oi >> 1, i = oi & 1;
    const int r = (int)(q % orr);
    double v = 0.0;
    const bool ul_in = first ? true : l < ul;
    const bool ur_in = last ? true : r < ur;
    if (ul_in && ur_in) {
      const int lu = first ? 0 : l, ru = last ? 0 : r;
      v = U[((size_t)lu * 4 + oi) * ur + ru];
    }
    const bool tl_in = first ? true : l >= ul;
    const bool tr_in = last ? true : r >= ur;
    if (tl_in && tr_in) {
      const int lt = first ? 0 : l - ul, rt = last ? 0 : r - ur;
      (void)tl;
      (void)tr;
      if (e.is_x) {
        // (ea, d) -> (eb, d'):  E[ea][o][eb] delta_oi delta_dd'
        const int ea = lt / e.dw, da = lt % e.dw, eb = rt / e.dw, db = rt % e.dw;
        if (o == i && da == db) v += e.Ecore[((size_t)ea * 2 + o) * e.er + eb];
      } else {
        // (ea, da) -> (eb, db):  delta_ea,eb D[da][o][i][db]
        const int ea = lt / e.dl, da = lt % e.dl, eb = rt / e.dr, db = rt % e.dr;
        if (ea == eb) v += e.Dcore[((size_t)da * 4 + oi) * e.dr + db];
      }
    }
    out[q] = v;
  }
}
__global__ void k_assemble(const double* __restrict__ U, int ul, int ur, ETermSite e, int first, int last,
                           double* __restrict__ out, int ol, int orr) { k_assemble_body(U, ul, ur, e, first, last, out, ol, orr); }

int launch_assemble_site(vp_ctx* ctx, const double* U, int ul, int ur, const ETermSite& e, int first, int last,
                         double* out, int ol, int orr) {
  const size_t total = (size_t)ol * 4 * orr;
  ctx->launches++;
  k_assemble<<<grid_for(ctx, total), 256, 0, ctx->stream>>>(U, ul, ur, e, first, last, out, ol, orr);
  return check_launch(ctx, "assemble");
}

// Dense MPO contraction step (tests): T (rows x w) with rows = (out, in)
// pairs of the sites so far, times core (w, 2, 2, wr) -> (rows*4 x wr) with
// the new (out, in) bits appended: new row index = ((o_prev*2+o) , (i_prev*2+i)).
__global__ void k_mpo_dense_step(const double* __restrict__ T, int nrow_o, int w, const double* __restrict__ core,
                                 int wr, double* __restrict__ out) {
  // T layout: [o_prev][i_prev][w], o_prev, i_prev in [0, nrow_o)
  const size_t no = (size_t)nrow_o * 2;
  const size_t total = no * no * wr;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const size_t oo = q / (no * wr), ii = (q / wr) % no;
    const int r = (int)(q % wr);
    const size_t op = oo >> 1, ip = ii >> 1;
    const int o = (int)(oo & 1), i = (int)(ii & 1);
    double acc = 0.0;
    for (int a = 0; a < w; ++a)
      acc += T[(op * nrow_o + ip) * w + a] * core[((size_t)a * 4 + o * 2 + i) * wr + r];
    out[q] = acc;
  }
}

int launch_mpo_dense_step(vp_ctx* ctx, const double* T, int rows, int cols, int w, const double* core, int wr,
                          double* out) {
  (void)cols;
  const size_t no = (size_t)rows * 2;
  ctx->launches++;
  k_mpo_dense_step<<<grid_for(ctx, no * no * wr), 256, 0, ctx->stream>>>(T, rows, w, core, wr, out);
  return check_launch(ctx, "mpo_dense");
}

// Input check: any NaN or Inf among n values sets the status error 2 (the
// factorisations do not propagate every NaN: a column whose norm is NaN forms
// no reflector, so a corrupt input must be caught before them).
__device__ __forceinline__ void k_check_finite_body(const double* __restrict__ x, size_t n, DevStatus* st) {
  bool bad = false;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    bad |= !isfinite(x[e]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(&st->err, 0, 2);
}
__global__ void k_check_finite(const double* __restrict__ x, size_t n, DevStatus* st) { k_check_finite_body(x, n, st); }

int launch_check_finite(vp_ctx* ctx, const double* x, size_t n) {
  if (n == 0) return VP_OK;
  ctx->launches++;
  k_check_finite<<<grid_for(ctx, n), 256, 0, ctx->stream>>>(x, n, ctx->status);
  return check_launch(ctx, "check_finite");
}

// Sum of squared differences of two vectors, in a fixed order: per-block
// partial sums (grid-stride), then one block adds the partials in block
// order (deterministic, unlike atomics).
__global__ void k_sqdiff_partial(const double* __restrict__ a, const double* __restrict__ b, size_t n,
                                 double* __restrict__ part) {
  __shared__ double red[32];
  double acc = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double d = a[e] - b[e];
    acc = fma(d, d, acc);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}
__global__ void k_sum_partials(const double* __restrict__ part, int nb, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < nb; ++i) t += part[i];
    *out = t;
  }
}

int launch_sqdiff(vp_ctx* ctx, const double* a, const double* b, size_t n, double* scratch, double* out) {
  const int blocks = std::min(1024, grid_for(ctx, n));
  ctx->launches += 2;
  k_sqdiff_partial<<<blocks, 256, 0, ctx->stream>>>(a, b, n, scratch);
  VP_TRY(check_launch(ctx, "sqdiff"));
  k_sum_partials<<<1, 32, 0, ctx->stream>>>(scratch, blocks, out);
  return check_launch(ctx, "sum_partials");
}

// ====================================================== batched launches
// (see common.cuh): the body of each single-problem kernel for the problem the
// grid's y coordinate selects, with that problem's own x extent.
namespace {
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
}  // namespace

__global__ void kb_check_finite(const __grid_constant__ Pack<BCheck> pk) {
  const BCheck& a = pk.a[blockIdx.y];
  k_check_finite_body(a.x, a.n, a.st);
}
int blaunch_check_finite(vp_ctx* ctx, cudaStream_t st, const std::vector<BCheck>& v) {
  return run_packs(ctx, st, v, kb_check_finite, 256, 0, [&](const BCheck& a) { return grid_for(ctx, a.n); },
                   "b_check_finite");
}
__global__ void kb_copy(const __grid_constant__ Pack<BCopy> pk) {
  const BCopy& a = pk.a[blockIdx.y];
  k_copy_body(a.src, a.dst, a.n);
}
int blaunch_copy(vp_ctx* ctx, cudaStream_t st, const std::vector<BCopy>& v) {
  std::vector<BCopy> nz;
  for (const BCopy& c : v)
    if (c.n) nz.push_back(c);
  return run_packs(ctx, st, nz, kb_copy, 256, 0, [&](const BCopy& a) { return grid_for(ctx, a.n); }, "b_copy");
}
__global__ void kb_site_sum(const __grid_constant__ Pack<BSiteSum> pk) {
  const BSiteSum& a = pk.a[blockIdx.y];
  k_site_sum_body(a.s, a.out, a.ol, a.orr);
}
int blaunch_site_sum(vp_ctx* ctx, cudaStream_t st, const std::vector<BSiteSum>& v) {
  return run_packs(ctx, st, v, kb_site_sum, 256, 0,
                   [&](const BSiteSum& a) { return grid_for(ctx, (size_t)a.ol * 2 * a.orr); }, "b_site_sum");
}
__global__ void kb_phys_sum(const __grid_constant__ Pack<BPhysSum> pk) {
  const BPhysSum& a = pk.a[blockIdx.y];
  k_phys_sum_body(a.core, a.rl, a.rr, a.T);
}
int blaunch_phys_sum(vp_ctx* ctx, cudaStream_t st, const std::vector<BPhysSum>& v) {
  return run_packs(ctx, st, v, kb_phys_sum, 256, 0,
                   [&](const BPhysSum& a) { return grid_for(ctx, (size_t)a.rl * a.rr); }, "b_phys_sum");
}
__global__ void kb_scale(const __grid_constant__ Pack<BScale> pk) {
  const BScale& a = pk.a[blockIdx.y];
  k_scale_body(a.x, a.n, a.s);
}
int blaunch_scale(vp_ctx* ctx, cudaStream_t st, const std::vector<BScale>& v) {
  std::vector<BScale> nz;
  for (const BScale& c : v)
    if (c.n) nz.push_back(c);
  return run_packs(ctx, st, nz, kb_scale, 256, 0, [&](const BScale& a) { return grid_for(ctx, a.n); }, "b_scale");
}
__global__ void kb_poisson(const __grid_constant__ Pack<BPoisson> pk) {
  const BPoisson& a = pk.a[blockIdx.y];
  k_poisson_body(a.rho, a.N, a.dx, a.E, a.we);
}
int blaunch_poisson(vp_ctx* ctx, cudaStream_t st, const std::vector<BPoisson>& v) {
  const int nt = 256;
  size_t smem = 0;
  for (const BPoisson& a : v) smem = std::max(smem, (size_t)(a.N + 33 + nt) * sizeof(double));
  if (smem > 200 * 1024) return fail(ctx, VP_ECAPACITY, "poisson: 2^nx too large");
  static AttrOnce at;
  VP_TRY(at.ensure(ctx, (const void*)kb_poisson, 200 * 1024, false));
  return run_packs(ctx, st, v, kb_poisson, nt, smem, [](const BPoisson&) { return 1; }, "b_poisson");
}
__global__ void kb_assemble(const __grid_constant__ Pack<BAssemble> pk) {
  const BAssemble& a = pk.a[blockIdx.y];
  k_assemble_body(a.U, a.ul, a.ur, a.e, a.first, a.last, a.out, a.ol, a.orr);
}
int blaunch_assemble(vp_ctx* ctx, cudaStream_t st, const std::vector<BAssemble>& v) {
  return run_packs(ctx, st, v, kb_assemble, 256, 0,
                   [&](const BAssemble& a) { return grid_for(ctx, (size_t)a.ol * 4 * a.orr); }, "b_assemble");
}
__global__ void kb_permute(const __grid_constant__ Pack<BPermute> pk) {
  const BPermute& a = pk.a[blockIdx.y];
  k_permute_body(a.f, a.nx, a.nv, a.mapping, a.out, a.inverse);
}
int blaunch_permute(vp_ctx* ctx, cudaStream_t st, const std::vector<BPermute>& v) {
  return run_packs(ctx, st, v, kb_permute, 256, 0,
                   [&](const BPermute& a) { return grid_for(ctx, (size_t)1 << (a.nx + a.nv)); }, "b_permute");
}

}  // namespace vp
