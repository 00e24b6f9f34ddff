// Eight-lanes-per-row helpers shared by the row kernels (hstep.cu, admm.cu).
//
// A factor row of rank k (padded to KP = 16, 32, 48 or 64; padded entries are
// zero) is held in registers by eight consecutive lanes: lane `sub` owns the
// entries l = sub + 8 e, e < KP / 8.  Products with a KP x KP matrix in shared
// memory take each entry from its owner lane by a shuffle, so the FMAs of a
// lane are independent of each other.
#pragma once

#include "common.cuh"

namespace enmf {
namespace lanes {

constexpr int LPR = 8;   // lanes per row
constexpr unsigned FULL = 0xffffffffu;

template <typename T>
__device__ __forceinline__ T shfl8(T v, int src) {
  return __shfl_sync(FULL, v, src, LPR);
}

// Sum over the eight lanes of a row.  The butterfly gives every lane the same
// bits: each step adds a pair whose order only commutes.
template <typename T>
__device__ __forceinline__ T sum8(T v) {
  v += __shfl_xor_sync(FULL, v, 4, LPR);
  v += __shfl_xor_sync(FULL, v, 2, LPR);
  v += __shfl_xor_sync(FULL, v, 1, LPR);
  return v;
}

template <typename TF, int E>
__device__ __forceinline__ void load_row(const TF* P, int64_t i, bool live, int k, int sub,
                                         TF (&v)[E]) {
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int l = sub + LPR * e;
    v[e] = (live && l < k) ? P[i * k + l] : TF(0);
  }
}

template <typename TF, int E>
__device__ __forceinline__ void store_row(TF* P, int64_t i, bool live, int k, int sub,
                                          const TF (&v)[E]) {
  if (!live) return;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int l = sub + LPR * e;
    if (l < k) P[i * k + l] = v[e];
  }
}

// s_l = sum_m u_m Ms[m][l] for the lane's entries l (Ms: KP x KP row-major in
// shared memory), m in increasing order; u_m comes from its owner lane.
template <typename TF, int KP>
__device__ __forceinline__ void row_times(const TF* Ms, const TF (&u)[KP / LPR], int k, int sub,
                                          TF (&s)[KP / LPR]) {
  constexpr int E = KP / LPR;
#pragma unroll
  for (int e = 0; e < E; ++e) s[e] = TF(0);
#pragma unroll
  for (int m = 0; m < KP; ++m) {
    if (m < k) {
      const TF um = shfl8(u[m / LPR], m % LPR);
#pragma unroll
      for (int e = 0; e < E; ++e) s[e] = fma(um, Ms[m * KP + sub + LPR * e], s[e]);
    }
  }
}

// Adds sum over the block's staged rows of x_row^T y_row to the thread's
// (KP/16) x (KP/16) sub-block (bi, bj) = (thread / 16, thread % 16) of a
// KP x KP product, for a block of 256 threads; xs and ys hold `nrows` rows of
// KP entries.  The caller stages the rows and synchronises.
template <typename TF, int KP>
__device__ __forceinline__ void accumulate_outer(const TF* xs, const TF* ys, int nrows,
                                                 TF (&acc)[KP / 16][KP / 16]) {
  constexpr int S = KP / 16;
  const int bi = threadIdx.x / 16, bj = threadIdx.x % 16;
  for (int rr = 0; rr < nrows; ++rr) {
    TF x[S], y[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      x[s] = xs[rr * KP + bi * S + s];
      y[s] = ys[rr * KP + bj * S + s];
    }
#pragma unroll
    for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) acc[s1][s2] = fma(x[s1], y[s2], acc[s1][s2]);
  }
}

// out[e] = sum over the nb blocks of part[b * kk + e] (FP64 partials written
// before a grid barrier), for e < kk, one warp per entry, spread over blocks
// first .. gridDim.x - 1 (block 0 may be left free for other work): lane l
// takes partials l + 32 j in eight independent loads, then the eight are
// combined pairwise and the lanes by a butterfly.  The order is fixed by nb,
// so the sum does not depend on timing.  Block of BT threads.
// Entry e of the sum of nb block partials (part[b * kk + e]) by one warp, in
// a fixed order whoever runs it; every lane returns the total.
__device__ __forceinline__ double warp_sum_partials(const double* part, int nb, int kk, int e,
                                                   int lane) {
  double s = 0.0;
  for (int b0 = 0; b0 < nb; b0 += 256) {
    double c[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int b = b0 + lane + 32 * j;
      c[j] = b < nb ? __ldcg(&part[(int64_t)b * kk + e]) : 0.0;
    }
    s += ((c[0] + c[1]) + (c[2] + c[3])) + ((c[4] + c[5]) + (c[6] + c[7]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
  return s;
}

// The reduction runs on blocks bid = first .. nblk - 1 of a group of nblk
// blocks (by default the whole grid).
template <int BT>
__device__ __forceinline__ void sum_block_partials(const double* part, int nb, int kk,
                                                   double* out, int first = 0, int bid = -1,
                                                   int nblk = -1) {
  constexpr int WPB = BT / 32;
  if (bid < 0) {
    bid = (int)blockIdx.x;
    nblk = (int)gridDim.x;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nbk = nblk - first;
  if (bid < first || nbk <= 0) return;
  for (int e = (bid - first) * WPB + warp; e < kk; e += nbk * WPB) {
    const double s = warp_sum_partials(part, nb, kk, e, lane);
    if (lane == 0) out[e] = s;
  }
}

// Sum over a block of 256 threads with two barriers: a butterfly within each
// warp (every lane gets the same bits), then the eight warp sums in warp
// order.  Every thread returns the total; `sh` needs 8 doubles.
__device__ __forceinline__ double block_sum256(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  __syncthreads();   // sh free from any previous use
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  return ((sh[0] + sh[1]) + (sh[2] + sh[3])) + ((sh[4] + sh[5]) + (sh[6] + sh[7]));
}

// Two such sums at once (each in the order of block_sum256): a and b come
// back as the totals in every thread.  `sh` needs 16 doubles.
__device__ __forceinline__ void block_sum256x2(double& a, double& b, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(FULL, a, o);
    b += __shfl_xor_sync(FULL, b, o);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    sh[threadIdx.x >> 5] = a;
    sh[8 + (threadIdx.x >> 5)] = b;
  }
  __syncthreads();
  a = ((sh[0] + sh[1]) + (sh[2] + sh[3])) + ((sh[4] + sh[5]) + (sh[6] + sh[7]));
  b = ((sh[8] + sh[9]) + (sh[10] + sh[11])) + ((sh[12] + sh[13]) + (sh[14] + sh[15]));
}

// The same in FP32 (for sums whose FP32 rounding is far below what they are
// compared with -- the FP64 adds of all 256 threads cost more than the data
// warrants at this GPU's FP64 rate).  `sh` needs 8 floats.
__device__ __forceinline__ float block_sum256f(float v, float* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  return ((sh[0] + sh[1]) + (sh[2] + sh[3])) + ((sh[4] + sh[5]) + (sh[6] + sh[7]));
}

inline int rank_pad16(int k) { return k <= 16 ? 16 : (k <= 32 ? 32 : (k <= 48 ? 48 : 64)); }

}  // namespace lanes
}  // namespace enmf
