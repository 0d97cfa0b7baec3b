// vp_poisson_noalloc: the periodic Poisson field solve for callers that cannot
// allocate device memory.
//
// vp_poisson needs a vp_ctx, and creating a context allocates (status words,
// scratch, pinned mirrors).  Some callers cannot do that: code running inside
// another framework's memory budget with allocation disabled, a host thread
// that must not touch the allocator while a CUDA graph is being captured
// elsewhere, or an embedding whose device memory is fully reserved up front.
// This entry point takes only caller-owned buffers; its scratch (the prefix
// sums and the two reduced scalars) lives in a file-scope __device__ array
// that every GPU which loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/vpmps.h"

namespace {

constexpr int kMaxN = 1 << 14;  // largest grid: nx <= 14 (16384 points)
constexpr int kMaxDevices = 64;

// d[0 .. kMaxN) holds phi differences, [kMaxN, kMaxN + 2) the field energy and
// the mass.  Shared by every call on a device: concurrent calls race.
__device__ __align__(256) double g_poisson_scratch[kMaxN + 64];

double* g_scratch_addr[kMaxDevices] = {};
std::mutex g_setup_mutex;

__device__ __forceinline__ double bsum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w];
    red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// Same arithmetic as the context-based solve: s_i = dx^2 (rho_i - mean),
// d_i = phi_{i+1} - phi_i = d_0 + sum_{j=1}^{i} s_j with sum_i d_i = 0, and
// E_i = -(d_i + d_{i-1}) / (2 dx); d lives in the device scratch.
__global__ void k_poisson_noalloc(const double* __restrict__ rho, int N, double dx, double* __restrict__ E,
                                  double* __restrict__ d, double* __restrict__ out2) {
  __shared__ double red[33];
  __shared__ double part[256];
  const int tid = threadIdx.x, nt = blockDim.x;
  double loc = 0.0;
  for (int i = tid; i < N; i += nt) loc += rho[i];
  const double total = bsum(loc, red);
  const double mean = total / N;
  const int chunk = (N + nt - 1) / nt;
  const int lo = min(N, tid * chunk), hi = min(N, lo + chunk);
  double run = 0.0;
  for (int i = lo; i < hi; ++i) {
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
  const double d0 = -bsum(sS, red) / N;
  __syncthreads();
  for (int i = tid; i < N; i += nt) d[i] += d0;
  __syncthreads();
  double e2 = 0.0;
  for (int i = tid; i < N; i += nt) {
    const double e = -(d[i] + d[(i + N - 1) % N]) / (2.0 * dx);
    E[i] = e;
    e2 = fma(e, e, e2);
  }
  const double we = bsum(e2, red);
  if (tid == 0) {
    out2[0] = 0.5 * we * dx;
    out2[1] = total * dx;
  }
}

// Device address of the scratch for the current device, looked up once per
// device (cudaGetSymbolAddress with that device current).
int scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return VP_ECUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    double* p = nullptr;
    if (cudaGetSymbolAddress((void**)&p, g_poisson_scratch) != cudaSuccess || !p) return VP_ECUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return VP_OK;
}

}  // namespace

extern "C" int vp_poisson_noalloc(void* cuda_stream, const double* rho_dev, int nx, double dx, double* E_dev,
                                  double* field_energy_host, double* mass_host) {
  if (!rho_dev || !E_dev || nx < 1 || !(dx > 0)) return VP_EINVAL;
  if (nx > 14) return VP_ECAPACITY;  // 2^nx beyond the static scratch (16384 points)
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // the scratch address is the current device's: the stream must be on it
  int cur = 0, sdev = 0;
  if (cudaGetDevice(&cur) != cudaSuccess || cudaStreamGetDevice(st, &sdev) != cudaSuccess) return VP_ECUDA;
  if (sdev != cur) return VP_EINVAL;
  double* scratch = nullptr;
  const int s = scratch_for_current_device(&scratch);
  if (s != VP_OK) return s;
  k_poisson_noalloc<<<1, 256, 0, st>>>(rho_dev, 1 << nx, dx, E_dev, scratch, scratch + kMaxN);
  if (cudaGetLastError() != cudaSuccess) return VP_ECUDA;
  if (field_energy_host || mass_host) {
    double two[2];
    if (cudaMemcpyAsync(two, scratch + kMaxN, sizeof(two), cudaMemcpyDeviceToHost, st) != cudaSuccess) return VP_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return VP_ECUDA;
    if (field_energy_host) *field_energy_host = two[0];
    if (mass_host) *mass_host = two[1];
  }
  return VP_OK;
}
