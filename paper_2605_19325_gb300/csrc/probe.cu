// Measurement helpers of the library: an FMA-throughput probe (the FP64 and
// FP32 ALU peaks that bound the SIMT sweeps) and the launch counter.
#include <atomic>

#include "internal.h"

namespace enmf {

std::atomic<long long> g_launches{0};

void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// 8 independent FMA chains per thread; 2 flops per FMA.
template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T* out, int iters, T a, T b) {
  T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  T x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == T(-1)) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
}

}  // namespace enmf

using namespace enmf;

// Peak FMA throughput of this device in flop/s for dtype ENMF_F64 or
// ENMF_F32, timed with CUDA events on the legacy stream.
extern "C" enmf_status enmf_probe_fma_peak(int32_t dtype, double* flops_per_s) {
  if (!flops_per_s || (dtype != ENMF_F64 && dtype != ENMF_F32)) return ENMF_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ENMF_ECUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8, threads = 256;
  const int iters = dtype == ENMF_F64 ? 64 : 2048;
  void* out = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * threads * 8) != cudaSuccess) return ENMF_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0, 0);
    if (dtype == ENMF_F64)
      fma_probe_kernel<double><<<blocks, threads>>>((double*)out, iters, 0.999999, 1e-7);
    else
      fma_probe_kernel<float><<<blocks, threads>>>((float*)out, iters, 0.9999f, 1e-4f);
    cudaEventRecord(e1, 0);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (cudaGetLastError() != cudaSuccess) return ENMF_ECUDA;
  double flops = 2.0 * 8.0 * 16.0 * (double)iters * blocks * threads;
  *flops_per_s = flops / (best * 1e-3);
  return ENMF_OK;
}

// Kernel launches issued by the library since it was loaded.
extern "C" long long enmf_launch_count(void) { return g_launches.load(); }
