// Allocation-free residual: f = 1/2 ||X - U V^T||_F^2, the relative error
// and ||X||_F^2 (the three numbers enmf_residual returns with direct = 1),
// formed entry by entry, for callers that hold no
// context and must not allocate device memory.  Its reduction scratch is a
// fixed array in the library's static device memory, so the call makes no
// allocation of any kind.
//
// Work split: block b owns rows [64 b, 64 b + 64) of X (a "panel") and forms
// every entry x_ij - u_i . v_j of that panel exactly as the context path does
// (the dot product in the factors' type, fused multiply-adds in column order,
// the difference and its square in FP64).  It also sums x_ij^2, so X is read
// once.  Each block writes its two FP64 panel sums to the scratch; the last
// block to arrive (an arrival counter in the scratch) sums the panels in panel
// order and writes f, the relative error and ||X||_F^2 to the caller's device
// buffer.  Results are deterministic; they differ from enmf_residual only in
// the order of the FP64 sums.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include <atomic>
#include <mutex>

#include "internal.h"

namespace enmf {
namespace {

constexpr int NA_THREADS = 64;      // one column of a 64-column tile per thread
constexpr int NA_STAGE_ROWS = 16;   // rows of U staged in shared memory at once
constexpr int NA_PANEL = 64;        // rows of X per block
constexpr int NA_MAX_PANELS = ENMF_RESIDUAL_NOALLOC_MAX_ROWS / NA_PANEL;
static_assert(NA_MAX_PANELS * NA_PANEL == ENMF_RESIDUAL_NOALLOC_MAX_ROWS, "panel split");
constexpr int NA_MAX_DEVICES = 64;

// Scratch layout (doubles): [0, P) residual panel sums, [P, 2P) ||X||^2 panel
// sums, slot 2P the arrival counter (as a 64-bit integer), rest padding.
constexpr int NA_COUNTER = 2 * NA_MAX_PANELS;
constexpr int NA_SCRATCH_DOUBLES = 2 * NA_MAX_PANELS + 32;  // 65,792 bytes

}  // namespace
}  // namespace enmf

// The call's only scratch: one copy per device, in static device memory.
static __device__ __align__(256) double g_noalloc_scratch[enmf::NA_SCRATCH_DOUBLES];

namespace enmf {
namespace {

template <typename TX, typename TF>
__global__ void __launch_bounds__(NA_THREADS)
residual_noalloc_kernel(const TX* __restrict__ X, int64_t m, int64_t n, int64_t ldx,
                        const TF* __restrict__ U, const TF* __restrict__ V, int r,
                        double* __restrict__ scratch, double* __restrict__ out3) {
  __shared__ TF Us[NA_STAGE_ROWS][RMAX];
  __shared__ TF Vs[RMAX][NA_THREADS + 1];
  __shared__ double sh[NA_THREADS];
  __shared__ int last;
  const int64_t r0 = (int64_t)blockIdx.x * NA_PANEL, r1 = min(m, r0 + NA_PANEL);
  double se = 0.0, sx = 0.0;
  for (int64_t i0 = r0; i0 < r1; i0 += NA_STAGE_ROWS) {
    const int nr = (int)min((int64_t)NA_STAGE_ROWS, r1 - i0);
    __syncthreads();
    for (int e = threadIdx.x; e < NA_STAGE_ROWS * r; e += NA_THREADS) {
      const int rr = e / r, cc = e % r;
      Us[rr][cc] = rr < nr ? U[(i0 + rr) * r + cc] : TF(0);
    }
    for (int64_t j0 = 0; j0 < n; j0 += NA_THREADS) {
      const int nc = (int)min((int64_t)NA_THREADS, n - j0);
      __syncthreads();
      for (int e = threadIdx.x; e < NA_THREADS * r; e += NA_THREADS) {
        const int jj = e / r, cc = e % r;
        Vs[cc][jj] = jj < nc ? V[(j0 + jj) * r + cc] : TF(0);
      }
      __syncthreads();
      const int jj = threadIdx.x;
      if (jj < nc) {
        for (int rr = 0; rr < nr; ++rr) {
          TF dotv = TF(0);
          for (int c = 0; c < r; ++c) dotv = fma(Us[rr][c], Vs[c][jj], dotv);
          const double x = to_d(X[(i0 + rr) * ldx + j0 + jj]);
          const double e = x - (double)dotv;
          se = fma(e, e, se);
          sx = fma(x, x, sx);
        }
      }
    }
  }
  se = block_sum(se, sh);
  sx = block_sum(sx, sh);
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(&scratch[NA_COUNTER]);
  if (threadIdx.x == 0) {
    scratch[blockIdx.x] = se;
    scratch[NA_MAX_PANELS + blockIdx.x] = sx;
    __threadfence();
    last = atomicAdd(counter, 1ULL) == (unsigned long long)(gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // Panel sums in panel order: thread t takes panels t, t + 64, ..., then a
  // fixed-tree block sum.
  double te = 0.0, tx = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += NA_THREADS) {
    te += __ldcg(&scratch[b]);
    tx += __ldcg(&scratch[NA_MAX_PANELS + b]);
  }
  te = block_sum(te, sh);
  tx = block_sum(tx, sh);
  if (threadIdx.x == 0) {
    out3[0] = 0.5 * te;
    out3[1] = tx > 0.0 ? sqrt(te > 0.0 ? te : 0.0) / sqrt(tx) : 0.0;
    out3[2] = tx;
    *counter = 0ULL;
  }
}

// Per-device scratch address, resolved once with that device current.
std::atomic<double*> g_scratch_addr[NA_MAX_DEVICES];
std::mutex g_setup_mu;

template <typename TX, typename TF>
cudaError_t load_kernel() {
  cudaFuncAttributes a;
  return cudaFuncGetAttributes(&a, residual_noalloc_kernel<TX, TF>);
}

// First call on a device: look up the scratch array's device address and load
// every instantiation of the kernel, so that later calls only enqueue work.
enmf_status scratch_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return ENMF_ECUDA;
  }
  if (dev < 0 || dev >= NA_MAX_DEVICES) return ENMF_EINVAL;
  double* p = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (p) {
    *out = p;
    return ENMF_OK;
  }
  std::lock_guard<std::mutex> lock(g_setup_mu);
  p = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!p) {
    double* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch);
    if (e == cudaSuccess) e = load_kernel<double, double>();
    if (e == cudaSuccess) e = load_kernel<float, float>();
    if (e == cudaSuccess) e = load_kernel<__nv_bfloat16, float>();
    if (e == cudaSuccess) e = load_kernel<__half, float>();
    if (e != cudaSuccess || !ptr) {
      cudaGetLastError();
      return ENMF_ECUDA;
    }
    p = ptr;
    g_scratch_addr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return ENMF_OK;
}

}  // namespace
}  // namespace enmf

using namespace enmf;

extern "C" enmf_status enmf_residual_noalloc(const void* X, int32_t x_dtype, int64_t m, int64_t n,
                                            int64_t ldx, const void* U, const void* V, int32_t r,
                                            int32_t f_dtype, double* out3, void* stream) {
  if (!out3) return ENMF_EINVAL;
  if (m < 0 || n < 0 || ldx < n) return ENMF_EINVAL;
  if (m > ENMF_RESIDUAL_NOALLOC_MAX_ROWS) return ENMF_EINVAL;
  if (r < 1 || r > ENMF_MAX_RANK) return ENMF_EINVAL;
  if (x_dtype < ENMF_F64 || x_dtype > ENMF_F16) return ENMF_EINVAL;
  if (f_dtype == ENMF_F64 ? x_dtype != ENMF_F64 : f_dtype != ENMF_F32) return ENMF_EINVAL;
  if (m > 0 && n > 0 && (!X || !U || !V)) return ENMF_EINVAL;
  double* scratch = nullptr;
  enmf_status rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (m == 0 || n == 0) {
    // Empty X: f = 0, relative error 0, ||X||^2 = 0.
    if (cudaMemsetAsync(out3, 0, 3 * sizeof(double), s) != cudaSuccess) {
      cudaGetLastError();
      return ENMF_ECUDA;
    }
    return ENMF_OK;
  }
  // The arrival counter must start at zero.
  if (cudaMemsetAsync(&scratch[NA_COUNTER], 0, sizeof(unsigned long long), s) != cudaSuccess) {
    cudaGetLastError();
    return ENMF_ECUDA;
  }
  const int grid = (int)((m + NA_PANEL - 1) / NA_PANEL);
  note_launch(1);
#define NA_LAUNCH(TX, TF)                                                                  \
  residual_noalloc_kernel<TX, TF><<<grid, NA_THREADS, 0, s>>>(                             \
      (const TX*)X, m, n, ldx, (const TF*)U, (const TF*)V, r, scratch, out3)
  if (x_dtype == ENMF_F64) NA_LAUNCH(double, double);
  else if (x_dtype == ENMF_F32) NA_LAUNCH(float, float);
  else if (x_dtype == ENMF_BF16) NA_LAUNCH(__nv_bfloat16, float);
  else NA_LAUNCH(__half, float);
#undef NA_LAUNCH
  if (cudaGetLastError() != cudaSuccess) return ENMF_ECUDA;
  return ENMF_OK;
}
