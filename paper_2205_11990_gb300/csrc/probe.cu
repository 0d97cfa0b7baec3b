// Arithmetic-rate probes (vp_peak_probe): the throughput of the units the
// factorisations and contractions run on, measured on this device with
// enough independent chains per thread and warps per SM to hide latency.
// They set no device state; each probe is one timed launch after one warm-up
// launch on the context's stream.
//
//   FP64 FMA      fma(double) chains: 2 flops each (the FP64 pipe)
//   FP32 FMA      fmaf chains: 2 flops each
//   DW dot step   one step of the compensated double-word dot product
//                 (12 FP32 instructions, 2 FP64-equivalent flops)
//   DW axpy       one element of c <- c - w v in double words (29 FP32
//                 instructions, 2 FP64-equivalent flops)
//   DMMA          mma.sync m8n8k4 FP64 on the tensor cores (512 flops per
//                 warp instruction)
#include <cuda_runtime.h>

#include "common.cuh"
#include "dw.cuh"

namespace vp {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) k_probe_fp64(double a, double b, int iters, double* out) {
  double acc[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) acc[j] = (double)(threadIdx.x + j);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int j = 0; j < kChains; ++j) acc[j] = fma(acc[j], a, b);
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += acc[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_fp32(float a, float b, int iters, double* out) {
  float acc[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) acc[j] = (float)(threadIdx.x + j);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int j = 0; j < kChains; ++j) acc[j] = fmaf(acc[j], a, b);
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += acc[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_dw_dot(float xh, float xl, int iters, double* out) {
  dw_acc acc[kChains];
  dw y[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) y[j] = {1.0f + 1e-3f * (threadIdx.x + j), 1e-9f};
  const dw x = {xh, xl};
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int j = 0; j < kChains; ++j) dw_dot_step(acc[j], x, y[j]);
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += dw_to(dw_acc_value(acc[j]));
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_dw_axpy(float wh, float wl, int iters, double* out) {
  dw c[kChains], v[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) {
    c[j] = {1.0f + 1e-3f * (threadIdx.x + j), 0.f};
    v[j] = {1e-6f * (j + 1), 1e-14f};
  }
  const dw w = {wh, wl};
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int j = 0; j < kChains; ++j) c[j] = dw_add(c[j], dw_neg(dw_mul(w, v[j])));
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += dw_to(c[j]);
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// One warp-wide m8n8k4 FP64 MMA: D (8x8) = A (8x4) B (4x8) + C; each lane holds
// one element of A and B and two of C/D.  Four independent accumulators.
__global__ void __launch_bounds__(kProbeThreads) k_probe_dmma(double a, double b, int iters, double* out) {
  double d0[4], d1[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    d0[j] = 0.0;
    d1[j] = 0.0;
  }
  const double av = a * (1 + (threadIdx.x & 3)), bv = b;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int j = 0; j < 4; ++j)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(d0[j]), "+d"(d1[j])
                   : "d"(av), "d"(bv));
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 4; ++j) s += d0[j] + d1[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace vp

using namespace vp;

extern "C" int vp_peak_probe(vp_ctx* ctx, int kind, double* tflops_out) {
  if (!ctx || !tflops_out || kind < VP_PROBE_FP64_FMA || kind > VP_PROBE_DMMA)
    return fail(ctx, VP_EINVAL, "vp_peak_probe: bad argument");
  const int blocks = ctx->num_sms * 4;  // 32 warps per SM
  const int threads = kProbeThreads;
  const int iters = kind == VP_PROBE_DW_AXPY ? 4096 : (kind == VP_PROBE_DMMA ? 2048 : 16384);
  double* out = (double*)dev_alloc(ctx, sizeof(double) * (size_t)blocks * threads);
  if (!out) return fail(ctx, VP_ENOMEM, "vp_peak_probe: device allocation failed");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int st = VP_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    st = fail(ctx, VP_ECUDA, "vp_peak_probe: event creation failed");
  float ms = 0.f;
  for (int rep = 0; rep < 2 && st == VP_OK; ++rep) {  // a warm-up launch, then the timed one
    cudaEventRecord(e0, ctx->stream);
    switch (kind) {
      case VP_PROBE_FP64_FMA: k_probe_fp64<<<blocks, threads, 0, ctx->stream>>>(1.0000001, 1e-9, iters, out); break;
      case VP_PROBE_FP32_FMA: k_probe_fp32<<<blocks, threads, 0, ctx->stream>>>(1.0000001f, 1e-9f, iters, out); break;
      case VP_PROBE_DW_DOT: k_probe_dw_dot<<<blocks, threads, 0, ctx->stream>>>(0.999f, 1e-10f, iters, out); break;
      case VP_PROBE_DW_AXPY: k_probe_dw_axpy<<<blocks, threads, 0, ctx->stream>>>(0.5f, 1e-9f, iters, out); break;
      default: k_probe_dmma<<<blocks, threads, 0, ctx->stream>>>(1e-3, 1e-3, iters, out); break;
    }
    ctx->launches++;
    cudaEventRecord(e1, ctx->stream);
    st = check_launch(ctx, "peak_probe");
    if (st == VP_OK && cudaEventSynchronize(e1) != cudaSuccess) st = fail(ctx, VP_ECUDA, "vp_peak_probe: sync failed");
    if (st == VP_OK) cudaEventElapsedTime(&ms, e0, e1);
  }
  if (st == VP_OK) {
    const double threads_total = (double)blocks * threads;
    double flops;
    if (kind == VP_PROBE_DMMA)
      flops = threads_total / 32.0 * iters * 4 * 512.0;
    else
      flops = threads_total * iters * kChains * 2.0;
    *tflops_out = flops / (ms * 1e-3) / 1e12;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  dev_free(ctx, out, sizeof(double) * (size_t)blocks * threads);
  return st;
}
