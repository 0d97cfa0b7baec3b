// Tensor-core contractions for the reduced-precision modes (tcgen05, TMEM,
// TMA).  The GEMM-shaped contractions of the sweeps (R times the next core,
// the absorbed U S products) run as C = alpha * A B with A (M x K) and B
// (K x N) given in FP64; the factorisations themselves stay FP64.
//
//   VP_PREC_TF32    operands rounded to TF32 (round to nearest), products
//                   accumulated in FP32 in tensor memory;
//   VP_PREC_BF16    operands rounded to BF16, FP32 accumulation;
//   VP_PREC_TF32X3  split products: a = a_hi + a_lo with a_hi = tf32(a),
//                   a_lo = tf32(a - a_hi), and A B ~ A_hi B_hi + A_hi B_lo +
//                   A_lo B_hi, FP32 accumulation.  The three products are one
//                   GEMM over a tripled K: A' = [A_hi | A_hi | A_lo],
//                   B' = [B_hi | B_lo | B_hi].
//
// Kernel: one CTA per 128 x BN output tile (BN = 64 or 128), four warps.
// Operands are packed K-major and zero-padded to whole tiles, so every TMA
// box is in bounds and 16-byte aligned.  Warp 0 lane 0 streams 128-byte-wide
// K blocks of A and B into a 4-stage shared-memory ring with
// cp.async.bulk.tensor (128-byte swizzle); warp 1 lane 0 issues
// tcgen05.mma (M = 128, N = BN, K = 32 bytes per instruction) into an FP32
// accumulator in tensor memory and releases each stage with tcgen05.commit;
// then all four warps read their 32 accumulator lanes with tcgen05.ld and
// write FP64 results.  Every wait is bounded (about 2 s); on a timeout the
// kernel flags the device status, lets its copies in flight land, frees its
// tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace vp {

namespace {

constexpr int kTcStages = 4;
constexpr uint32_t kTcABytes = 128 * 128;  // 128 rows x 128 bytes of K
constexpr long long kTcWaitNs = 2000000000ll;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Wait until the phase of parity `parity` has completed; false after ~2 s.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  const unsigned long long t0 = global_ns();
  for (long long it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 63) == 63 && global_ns() - t0 > (unsigned long long)kTcWaitNs) return false;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major tile written by TMA with the
// 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFF) >> 4);  // start address / 16
  d |= static_cast<uint64_t>(1) << 16;                  // leading byte offset (unused when swizzled K-major)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;          // stride byte offset: one 8-row group
  d |= static_cast<uint64_t>(1) << 46;                  // descriptor version
  d |= static_cast<uint64_t>(2) << 61;                  // 128-byte swizzle
  return d;
}

// Instruction descriptor: FP32 accumulator, A/B format `fmt` (TF32 = 2 with
// kind::tf32, BF16 = 1 with kind::f16), both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t tc_idesc(uint32_t fmt, int n) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | (static_cast<uint32_t>(n >> 3) << 17) | ((128u >> 4) << 24);
}

template <bool BF16>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (BF16) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  }
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <bool BF16, int BN>
__global__ void __launch_bounds__(128, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int M, int N,
              int kblocks, double alpha, double* __restrict__ C, int ldc, DevStatus* st) {
  constexpr uint32_t kB = BN * 128;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = base;
  uint8_t* sB = base + kTcStages * kTcABytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + kTcStages * kB);
  uint64_t* empty = full + kTcStages;
  uint64_t* done = empty + kTcStages;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ int s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * 128, n0 = blockIdx.x * BN;

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                 "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  bool ok = true;

  if (warp == 0 && lane == 0) {
    // producer: K blocks of A and B into the stage ring
    int last = -1;
    for (int kb = 0; kb < kblocks; ++kb) {
      const int s = kb % kTcStages;
      if (kb >= kTcStages && !mbar_wait(&empty[s], ((kb / kTcStages) - 1) & 1)) {
        ok = false;
        break;
      }
      mbar_expect_tx(&full[s], kTcABytes + kB);
      tma_load_2d(sA + s * kTcABytes, &ta, &full[s], kb * (BF16 ? 64 : 32), m0);
      tma_load_2d(sB + s * kB, &tb, &full[s], kb * (BF16 ? 64 : 32), n0);
      last = kb;
    }
    // every issued copy lands before the CTA can exit
    for (int s = 0; s < kTcStages; ++s) {
      const int kb = last - ((last - s) % kTcStages + kTcStages) % kTcStages;
      if (kb >= 0 && kb % kTcStages == s && !mbar_wait(&full[s], (kb / kTcStages) & 1)) ok = false;
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: four K steps of 32 bytes per 128-byte block
    constexpr uint32_t idesc = tc_idesc(BF16 ? 1u : 2u, BN);
    for (int kb = 0; kb < kblocks; ++kb) {
      const int s = kb % kTcStages;
      if (!mbar_wait(&full[s], (kb / kTcStages) & 1)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA + s * kTcABytes), b0 = smem_u32(sB + s * kB);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        tc_mma<BF16>(tmem, sw128_desc(a0 + 32 * k), sw128_desc(b0 + 32 * k), idesc, (kb | k) != 0 ? 1u : 0u);
      tc_commit(&empty[s]);
    }
    tc_commit(done);  // arrives once every MMA issued above has completed
  }
  if (!ok) atomicExch(&s_abort, 1);
  __syncwarp();
  __syncthreads();

  // epilogue: warp w owns accumulator lanes (rows) 32 w .. 32 w + 31; the
  // go/no-go decision is CTA-uniform, since tcgen05.ld is warp-collective
  const bool got = mbar_wait(done, 0);
  const int good = __syncthreads_and(got && s_abort == 0);
  tc_fence_after();
  if (good) {
    const int row = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      uint32_t r[16];
      tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0, r);
      if (row < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = n0 + c0 + j;
          if (col < N) C[(size_t)row * ldc + col] = alpha * static_cast<double>(__uint_as_float(r[j]));
        }
      }
    }
  }
  if (!good && threadIdx.x == 0) atomicCAS(&st->err, 0, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}

__device__ __forceinline__ double tc_elem(const TcOperand& o, int r, int k) {
  if (o.kind == 0) return o.p[(size_t)r * o.ld + k];
  if (o.kind == 1) return o.p[(size_t)k * o.ld + r];
  return r <= k ? o.p[(size_t)k * o.ld + r] : 0.0;
}

// Pack an R x K operand K-major into Rp x Kt (zero padded).  mode: 2 TF32,
// 3 BF16, 4 split TF32 with K tripled (role 0: hi, hi, lo; role 1: hi, lo, hi).
__global__ void k_tc_pack(TcOperand op, int R, int K, int Rp, int Kp, int mode, int role, void* out) {
  const size_t total = (size_t)Rp * Kp;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / Kp), k = (int)(e % Kp);
    const double v = (r < R && k < K) ? tc_elem(op, r, k) : 0.0;
    if (mode == 3) {
      reinterpret_cast<__nv_bfloat16*>(out)[e] = __float2bfloat16_rn(static_cast<float>(v));
    } else {
      const float hi = tf32_rna(static_cast<float>(v));
      if (mode == 2) {
        reinterpret_cast<float*>(out)[e] = hi;
      } else {
        const float lo = tf32_rna(static_cast<float>(v - static_cast<double>(hi)));
        float* row = reinterpret_cast<float*>(out) + (size_t)r * 3 * Kp;
        row[k] = hi;
        row[Kp + k] = role == 0 ? hi : lo;
        row[2 * Kp + k] = role == 0 ? lo : hi;
      }
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 2-D map over a K-major (rows x kt) buffer; box = 128 bytes of K x box_rows.
int make_map(vp_ctx* ctx, CUtensorMap* map, void* ptr, int rows, int kt, bool bf16, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return fail(ctx, VP_ECUDA, "tensor-core GEMM: cuTensorMapEncodeTiled unavailable");
  const size_t es = bf16 ? 2 : 4;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(kt), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(kt) * es};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(128 / es), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, ptr, dims,
                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ctx, VP_ECUDA, "tensor-core GEMM: tensor map encoding failed");
  return VP_OK;
}

size_t tc_smem_bytes(int bn) {
  return 1024 + kTcStages * (kTcABytes + (size_t)bn * 128) + (2 * kTcStages + 1) * 8 + 16;
}

template <bool BF16, int BN>
int launch_tc(vp_ctx* ctx, const CUtensorMap& ta, const CUtensorMap& tb, int M, int N, int kblocks, double alpha,
              double* C, int ldc) {
  static AttrOnce attr;  // per device
  VP_TRY(attr.ensure(ctx, (const void*)k_tc_gemm<BF16, BN>, (int)tc_smem_bytes(BN), false));
  dim3 grid((N + BN - 1) / BN, (M + 127) / 128);
  ctx->launches++;
  k_tc_gemm<BF16, BN><<<grid, 128, tc_smem_bytes(BN), ctx->stream>>>(ta, tb, M, N, kblocks, alpha, C, ldc,
                                                                      ctx->status);
  return check_launch(ctx, "tc_gemm");
}

int pack(vp_ctx* ctx, const TcOperand& op, int R, int K, int Rp, int Kp, int mode, int role, void* out) {
  const size_t total = (size_t)Rp * Kp;
  const int blocks = (int)std::min<size_t>((total + 255) / 256, (size_t)ctx->num_sms * 8);
  ctx->launches++;
  k_tc_pack<<<blocks, 256, 0, ctx->stream>>>(op, R, K, Rp, Kp, mode, role, out);
  return check_launch(ctx, "tc_pack");
}

}  // namespace

int launch_tc_gemm(vp_ctx* ctx, int M, int N, int K, double alpha, TcOperand a, TcOperand b, double* C, int ldc) {
  const int mode = ctx->precision;
  if (mode < VP_PREC_TF32 || mode > VP_PREC_TF32X3 || M <= 0 || N <= 0 || K <= 0)
    return fail(ctx, VP_EINVAL, "tensor-core GEMM: bad mode or shape");
  const bool bf16 = mode == VP_PREC_BF16;
  const int kel = bf16 ? 64 : 32;  // elements per 128-byte K block
  const size_t es = bf16 ? 2 : 4;
  const int bn = N <= 64 ? 64 : 128;
  const int Mp = (M + 127) / 128 * 128, Np = (N + bn - 1) / bn * bn, Kp = (K + kel - 1) / kel * kel;
  const int Kt = mode == VP_PREC_TF32X3 ? 3 * Kp : Kp;
  VP_TRY(reserve(ctx, ctx->w_tca, ((size_t)Mp * Kt * es + 7) / 8));
  VP_TRY(reserve(ctx, ctx->w_tcb, ((size_t)Np * Kt * es + 7) / 8));
  VP_TRY(pack(ctx, a, M, K, Mp, Kp, mode, 0, ctx->w_tca.p));
  VP_TRY(pack(ctx, b, N, K, Np, Kp, mode, 1, ctx->w_tcb.p));
  CUtensorMap ta, tb;
  VP_TRY(make_map(ctx, &ta, ctx->w_tca.p, Mp, Kt, bf16, 128));
  VP_TRY(make_map(ctx, &tb, ctx->w_tcb.p, Np, Kt, bf16, bn));
  const int kblocks = Kt / kel;
  if (bf16) {
    if (bn == 64) return launch_tc<true, 64>(ctx, ta, tb, M, N, kblocks, alpha, C, ldc);
    return launch_tc<true, 128>(ctx, ta, tb, M, N, kblocks, alpha, C, ldc);
  }
  if (bn == 64) return launch_tc<false, 64>(ctx, ta, tb, M, N, kblocks, alpha, C, ldc);
  return launch_tc<false, 128>(ctx, ta, tb, M, N, kblocks, alpha, C, ldc);
}

}  // namespace vp
