// Device helpers shared by the eNMF kernels: element conversion, fixed-order
// block reductions, a bounded grid-wide barrier for cooperative launches and a
// counter-based hash for the SVD start's test matrix.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace enmf {

// Device status word bits (the host maps them to enmf_status).
enum : int {
  ERR_TIMEOUT = 1,   // a bounded spin in a grid barrier expired
  ERR_NONFINITE = 2, // a non-finite value appeared
  ERR_NOTCONV = 4,   // Jacobi SVD did not converge / singular polar input
  ERR_DOMAIN = 8,    // negative entry in X
  ERR_FORMAT = 16,   // malformed compressed rows (pointers, column order or range)
};

constexpr int LMAX = 80;           // widest small matrix (r + oversample)
constexpr int RMAX = 64;           // widest factor (rank)
constexpr long long SPIN_BUDGET_CYCLES = 4000000000LL;  // ~2 s at 2 GHz

// ------------------------------------------- programmatic dependent launch
// A kernel launched as a programmatic dependent of the previous kernel on its
// stream may start while that kernel still runs; griddep_wait() returns once
// the previous kernel has completed and its writes are visible (at once when
// the kernel was launched without the attribute).  griddep_launch() lets the
// next kernel on the stream, if launched with the attribute, be scheduled
// early; every thread of a block calls it.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// --------------------------------------------------------------- conversion
template <typename T> __device__ __forceinline__ double to_d(T v);
template <> __device__ __forceinline__ double to_d<double>(double v) { return v; }
template <> __device__ __forceinline__ double to_d<float>(float v) { return (double)v; }
template <> __device__ __forceinline__ double to_d<__nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
template <> __device__ __forceinline__ double to_d<__half>(__half v) { return (double)__half2float(v); }

template <typename TO, typename TI> __device__ __forceinline__ TO cvt(TI v);
template <> __device__ __forceinline__ double cvt<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float cvt<float, double>(double v) { return (float)v; }
template <> __device__ __forceinline__ double cvt<double, float>(float v) { return (double)v; }
template <> __device__ __forceinline__ float cvt<float, float>(float v) { return v; }
template <> __device__ __forceinline__ float cvt<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ double cvt<double, __nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
template <> __device__ __forceinline__ float cvt<float, __half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ double cvt<double, __half>(__half v) { return (double)__half2float(v); }

// ------------------------------------------------------ fixed-order reduce
// Sum over the block in a fixed tree order (deterministic for a fixed
// blockDim).  `sh` needs blockDim.x doubles.  Result valid in thread 0 and
// returned to every thread.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  __syncthreads();
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  double out = sh[0];
  __syncthreads();
  return out;
}

__device__ __forceinline__ double block_max(double v, double* sh) {
  __syncthreads();
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  double out = sh[0];
  __syncthreads();
  return out;
}

__device__ __forceinline__ double block_min(double v, double* sh) {
  return -block_max(-v, sh);
}

// Max of nonnegative doubles through their bit patterns (order independent).
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr),
            (unsigned long long)__double_as_longlong(v));
}

// ------------------------------------------------------------ grid barrier
// Sense-by-generation barrier for cooperative launches (all blocks are
// co-resident).  The spin is bounded: on expiry the barrier records
// ERR_TIMEOUT in *err and lets the block continue, so no launch can hang.
// Grid-wide barrier state of the cooperative kernels (zero at creation).
struct GridBarrier {
  unsigned int word;
  unsigned int spin;   // spin limit in cycles; 0 = SPIN_BUDGET_CYCLES
};

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier of a cooperative launch, one atomic per block: block 0
// adds 2^31 - (nb - 1) and every other block adds 1, so over one barrier the
// word grows by exactly 2^31 -- bit 31 flips at the last arrival, whatever
// the order, and the low bits return to their value (any grid size may
// follow).  Thread 0 of each block arrives after a fence that publishes the
// block's writes (ordered by the preceding __syncthreads) and spins on an
// acquire load until bit 31 differs from the value its own atomic returned.
// The spin is bounded: past bar->spin cycles (SPIN_BUDGET_CYCLES when 0) it
// records ERR_TIMEOUT and the block goes on.
__device__ __forceinline__ void grid_sync(GridBarrier* bar, int* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
    const bool lead = blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0;
    const unsigned int inc = lead ? 0x80000000u - (nb - 1u) : 1u;
    const unsigned int lim = *(volatile unsigned int*)&bar->spin;
    const long long budget = lim ? (long long)lim : SPIN_BUDGET_CYCLES;
    __threadfence();
    const unsigned int old = atomicAdd(&bar->word, inc);
    const long long t0 = clock64();
    while (((ld_acquire_gpu(&bar->word) ^ old) & 0x80000000u) == 0u) {
      if (clock64() - t0 > budget) {
        atomicOr(err, ERR_TIMEOUT);
        break;
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// ------------------------------------------------------------- hash (RNG)
// splitmix64 finaliser on (seed, i, j) -> uniform double in (-1, 1).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double hash_uniform(uint64_t seed, uint64_t i, uint64_t j) {
  uint64_t h = mix64(seed ^ mix64(i * 0x100000001B3ull + mix64(j)));
  return ((double)(h >> 11) + 0.5) * (2.0 / 9007199254740992.0) - 1.0;
}

}  // namespace enmf
