// SIMT sweeps over X: X V and X^T U (App. I's core NMF kernel), the Grams and
// the FP64 reductions used for the objective of Eq. 1.
//
// These kernels serve the plain FP64 form and the FP32 form (and the SVD
// start of every form).  In FP64 they are bound by the DFMA rate, in FP32 by
// FFMA: at rank r one X element feeds 2r multiply-adds (X V and X^T U), so the
// arithmetic intensity is 4r / sizeof(X) flop per byte, far above the
// machine balance for both types.  Every output is computed by one thread in
// a fixed order and split-K partials are summed in a fixed order, so results
// are bitwise reproducible run to run.
#include "internal.h"

namespace enmf {

// ------------------------------------------------------------- tile shapes
template <typename TF> struct Tile;
template <> struct Tile<double> { static constexpr int BM = 32, BK = 32, KT = 32, TM = 2, TN = 4; };
template <> struct Tile<float>  { static constexpr int BM = 64, BK = 32, KT = 32, TM = 4, TN = 4; };

int choose_splits(int64_t rows_out, int64_t red_len, int k, int bm, int num_sms) {
  int64_t tiles = ((rows_out + bm - 1) / bm) * ((k + 31) / 32);
  int64_t target = 2LL * (num_sms > 0 ? num_sms : 152);
  int64_t splits = (target + tiles - 1) / tiles;
  int64_t max_by_len = red_len / 256;
  if (splits > max_by_len) splits = max_by_len;
  if (splits > 16) splits = 16;
  if (splits < 1) splits = 1;
  return (int)splits;
}

// C[rows_out x k] = op(X) * B, op = identity (TRANS=false: rows_out = m,
// reduction over n) or transpose (TRANS=true: rows_out = n, reduction over m).
// grid.x: output row tiles, grid.y: KT-wide column tiles, grid.z: K splits.
template <typename TX, typename TF, bool TRANS>
__global__ void __launch_bounds__((Tile<TF>::BM / Tile<TF>::TM) * (Tile<TF>::KT / Tile<TF>::TN))
sweep_kernel(const TX* __restrict__ X, int64_t m, int64_t n, int64_t ldx,
             const TF* __restrict__ B, int ldb, int k, TF* __restrict__ C, int ldc,
             int64_t red_per_split, TF* __restrict__ part) {
  constexpr int BM = Tile<TF>::BM, BK = Tile<TF>::BK, KT = Tile<TF>::KT;
  constexpr int TM = Tile<TF>::TM, TN = Tile<TF>::TN;
  constexpr int NR = BM / TM, NC = KT / TN, NT = NR * NC;
  __shared__ TF Xs[BK][BM + 1];
  __shared__ TF Bs[BK][KT];

  const int64_t rows_out = TRANS ? n : m;
  const int64_t red_len = TRANS ? m : n;
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const int col0 = blockIdx.y * KT;
  const int64_t kb = (int64_t)blockIdx.z * red_per_split;
  const int64_t ke = min(red_len, kb + red_per_split);
  const int tr = threadIdx.x / NC, tc = threadIdx.x % NC;

  TF acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = TF(0);

  for (int64_t k0 = kb; k0 < ke; k0 += BK) {
    if (!TRANS) {
      // X rows row0.., columns k0..: coalesced along the reduction index
      for (int e = threadIdx.x; e < BM * BK; e += NT) {
        int rr = e / BK, cc = e % BK;
        int64_t gr = row0 + rr, gc = k0 + cc;
        Xs[cc][rr] = (gr < m && gc < ke) ? cvt<TF>(X[gr * ldx + gc]) : TF(0);
      }
    } else {
      // X rows k0.., columns row0..: coalesced along the output index
      for (int e = threadIdx.x; e < BM * BK; e += NT) {
        int kk = e / BM, cc = e % BM;
        int64_t gr = k0 + kk, gc = row0 + cc;
        Xs[kk][cc] = (gr < ke && gc < n) ? cvt<TF>(X[gr * ldx + gc]) : TF(0);
      }
    }
    for (int e = threadIdx.x; e < BK * KT; e += NT) {
      int rr = e / KT, cc = e % KT;
      int64_t gr = k0 + rr;
      int gc = col0 + cc;
      Bs[rr][cc] = (gr < ke && gc < k) ? B[gr * ldb + gc] : TF(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < BK; ++kk) {
      TF a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = Xs[kk][tr + i * NR];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tc + j * NC];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int64_t gr = row0 + tr + i * NR;
    if (gr >= rows_out) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int gc = col0 + tc + j * NC;
      if (gc >= k) continue;
      if (part)
        part[((int64_t)blockIdx.z * rows_out + gr) * k + gc] = acc[i][j];
      else
        C[gr * ldc + gc] = acc[i][j];
    }
  }
}

// C = sum over splits of the partials, in split order.
template <typename TF>
__global__ void splitk_reduce(const TF* __restrict__ part, int splits, int64_t rows, int k,
                              TF* __restrict__ C, int ldc) {
  int64_t total = rows * k;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    TF s = part[e];
    for (int q = 1; q < splits; ++q) s += part[(int64_t)q * total + e];
    C[(e / k) * ldc + (e % k)] = s;
  }
}

template <typename TX, typename TF, bool TRANS>
static void sweep_launch(const void* X, int64_t m, int64_t n, int64_t ldx, const void* B, int ldb,
                         int k, void* C, int ldc, void* part, int num_sms, cudaStream_t s) {
  using T = Tile<TF>;
  int64_t rows_out = TRANS ? n : m, red = TRANS ? m : n;
  int splits = choose_splits(rows_out, red, k, T::BM, num_sms);
  int64_t per = (red + splits - 1) / splits;
  per = ((per + T::BK - 1) / T::BK) * T::BK;
  splits = (int)((red + per - 1) / per);
  dim3 grid((unsigned)((rows_out + T::BM - 1) / T::BM), (k + T::KT - 1) / T::KT, splits);
  int nt = (T::BM / T::TM) * (T::KT / T::TN);
  TF* p = splits > 1 ? (TF*)part : nullptr;
  note_launch(splits > 1 ? 2 : 1);
  sweep_kernel<TX, TF, TRANS><<<grid, nt, 0, s>>>((const TX*)X, m, n, ldx, (const TF*)B, ldb, k,
                                                  (TF*)C, ldc, per, p);
  if (splits > 1) {
    int64_t total = rows_out * k;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    splitk_reduce<TF><<<blocks, 256, 0, s>>>((const TF*)part, splits, rows_out, k, (TF*)C, ldc);
  }
}

// ------------------------------------------------ FP32-factor sweep (SIMT)
// C[rows_out x k] = op(X) B with FP32 factors and FP32 or 16-bit X (exact in
// FP32), FP32 products and sums.  One CTA owns BM output rows and KT columns
// over a range of the reduction: KT = 64 (BM = 128) for widths above 32 --
// every column of the SVD start's widths up to 64 in one pass over X -- and
// KT = 32 (BM = 256) up to 32, so that no FMA multiplies a padding column.
// 256 threads as (256 / (KT / 4)) x (KT / 4), thread (tr, tc) owning rows
// 8 tr .. 8 tr + 7 and columns 4 tc .. 4 tc + 3.  Stages of
// SW_BK reduction steps: the next stage's X and B values are loaded into
// registers while the current stage is multiplied out of shared memory (two
// buffers, one barrier per stage).  X sits in shared memory reduction-major.
// Per output the products are summed in reduction order, then the split-K
// partials in split order, so results are bitwise reproducible.
constexpr int SW_BK = 16, SW_T = 256;
__host__ __device__ constexpr int sw_bm(int kt) { return kt == 32 ? 256 : 128; }
static int sw_kt(int k) { return k <= 32 ? 32 : 64; }

int sweep_splits_f32(int64_t rows_out, int64_t red_len, int k, int num_sms) {
  const int kt = sw_kt(k), bm = sw_bm(kt);
  const int64_t tiles = ((rows_out + bm - 1) / bm) * ((k + kt - 1) / kt);
  const int64_t target = 2LL * (num_sms > 0 ? num_sms : 152);
  int64_t splits = (target + tiles - 1) / tiles;
  const int64_t max_by_len = red_len / 256;
  if (splits > max_by_len) splits = max_by_len;
  if (splits > 16) splits = 16;
  if (splits < 1) splits = 1;
  return (int)splits;
}

template <typename TX> struct Ld4;
template <> struct Ld4<float> {
  static __device__ __forceinline__ float4 vec(const float* p) { return *reinterpret_cast<const float4*>(p); }
};
template <> struct Ld4<__nv_bfloat16> {
  static __device__ __forceinline__ float4 vec(const __nv_bfloat16* p) {
    const uint2 u = *reinterpret_cast<const uint2*>(p);
    const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&u.x);
    const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&u.y);
    return make_float4(__low2float(a), __high2float(a), __low2float(b), __high2float(b));
  }
};
template <> struct Ld4<__half> {
  static __device__ __forceinline__ float4 vec(const __half* p) {
    const uint2 u = *reinterpret_cast<const uint2*>(p);
    const __half2 a = *reinterpret_cast<const __half2*>(&u.x);
    const __half2 b = *reinterpret_cast<const __half2*>(&u.y);
    return make_float4(__low2float(a), __high2float(a), __low2float(b), __high2float(b));
  }
};
__device__ __forceinline__ float ld1(const float* p) { return *p; }
__device__ __forceinline__ float ld1(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ float ld1(const __half* p) { return __half2float(*p); }

// Four consecutive entries p[0..3] of which those at offset >= lim read as 0
// (whole vector when VEC and all four are in range).
template <typename TX, bool VEC>
__device__ __forceinline__ float4 load4(const TX* p, int64_t lim) {
  if (VEC && lim >= 4) return Ld4<TX>::vec(p);
  float4 v;
  v.x = lim > 0 ? ld1(p) : 0.f;
  v.y = lim > 1 ? ld1(p + 1) : 0.f;
  v.z = lim > 2 ? ld1(p + 2) : 0.f;
  v.w = lim > 3 ? ld1(p + 3) : 0.f;
  return v;
}

template <typename TX, bool TRANS, bool VEC, int KT>
__global__ void __launch_bounds__(SW_T)
sweep32_kernel(const TX* __restrict__ X, int64_t m, int64_t n, int64_t ldx,
               const float* __restrict__ B, int ldb, int k, float* __restrict__ C, int ldc,
               int64_t red_per_split, float* __restrict__ part) {
  constexpr int BM = sw_bm(KT), BK = SW_BK, XLD = BM + 4;
  constexpr int TCN = KT / 4, TRN = SW_T / TCN;   // thread grid: TRN rows x TCN column groups
  constexpr int NV = BM * BK / 4 / SW_T;          // X float4s per thread per stage
  constexpr int BQ = BM / 4;                      // float4s across a reduction row (X^T U)
  static_assert(TRN * 8 == BM, "eight rows per thread");
  __shared__ __align__(16) float Xs[2][BK][XLD];
  __shared__ __align__(16) float Bs[2][BK][KT];
  const int t = threadIdx.x, tr = t / TCN, tc = t % TCN;
  const int64_t rows_out = TRANS ? n : m;
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const int col0 = blockIdx.y * KT;
  const int64_t kb = (int64_t)blockIdx.z * red_per_split;
  const int64_t ke = min(TRANS ? m : n, kb + red_per_split);

  float4 xr[NV], br;
  const bool bload = t < BK * TCN;   // threads holding one B float4 of a stage
  // global -> registers for the stage starting at k0
  auto fetch = [&](int64_t k0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int q = t + SW_T * v;
      if (!TRANS) {   // X rows row0 + q / 4, reduction columns k0 + 4 (q % 4) ..
        const int64_t gr = row0 + q / 4, gc = k0 + 4 * (q % 4);
        xr[v] = gr < m ? load4<TX, VEC>(X + gr * ldx + gc, ke - gc) : make_float4(0.f, 0.f, 0.f, 0.f);
      } else {        // X row k0 + q / BQ (reduction), columns row0 + 4 (q % BQ) ..
        const int64_t gr = k0 + q / BQ, gc = row0 + 4 * (q % BQ);
        xr[v] = gr < ke ? load4<TX, VEC>(X + gr * ldx + gc, n - gc) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    if (bload) {   // B rows k0 + t / TCN, columns col0 + 4 (t % TCN) ..
      const int64_t gr = k0 + t / TCN;
      const int gc = col0 + 4 * (t % TCN);
      br = gr < ke ? load4<float, VEC>(B + gr * ldb + gc, k - gc) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  auto stash = [&](int b) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int q = t + SW_T * v;
      if (!TRANS) {
        const int rr = q / 4, c4 = 4 * (q % 4);
        Xs[b][c4 + 0][rr] = xr[v].x;
        Xs[b][c4 + 1][rr] = xr[v].y;
        Xs[b][c4 + 2][rr] = xr[v].z;
        Xs[b][c4 + 3][rr] = xr[v].w;
      } else {
        *reinterpret_cast<float4*>(&Xs[b][q / BQ][4 * (q % BQ)]) = xr[v];
      }
    }
    if (bload) *reinterpret_cast<float4*>(&Bs[b][t / TCN][4 * (t % TCN)]) = br;
  };

  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

  int buf = 0;
  if (kb < ke) {
    fetch(kb);
    stash(0);
  }
  __syncthreads();
  for (int64_t k0 = kb; k0 < ke; k0 += BK) {
    const bool more = k0 + BK < ke;
    if (more) fetch(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      // the thread's eight rows are consecutive: two 16-byte loads
      const float4 a0 = *reinterpret_cast<const float4*>(&Xs[buf][kk][8 * tr]);
      const float4 a1 = *reinterpret_cast<const float4*>(&Xs[buf][kk][8 * tr + 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float4 b = *reinterpret_cast<const float4*>(&Bs[buf][kk][4 * tc]);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        acc[i][0] = fmaf(a[i], b.x, acc[i][0]);
        acc[i][1] = fmaf(a[i], b.y, acc[i][1]);
        acc[i][2] = fmaf(a[i], b.z, acc[i][2]);
        acc[i][3] = fmaf(a[i], b.w, acc[i][3]);
      }
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t gr = row0 + 8 * tr + i;
    if (gr >= rows_out) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gc = col0 + 4 * tc + j;
      if (gc >= k) continue;
      if (part)
        part[((int64_t)blockIdx.z * rows_out + gr) * k + gc] = acc[i][j];
      else
        C[gr * ldc + gc] = acc[i][j];
    }
  }
}

template <typename TX, bool TRANS>
static void sweep32_launch(const void* X, int64_t m, int64_t n, int64_t ldx, const void* B, int ldb,
                           int k, void* C, int ldc, void* part, int num_sms, cudaStream_t s) {
  const int64_t rows_out = TRANS ? n : m, red = TRANS ? m : n;
  int splits = sweep_splits_f32(rows_out, red, k, num_sms);
  int64_t per = (red + splits - 1) / splits;
  per = ((per + SW_BK - 1) / SW_BK) * SW_BK;
  splits = (int)((red + per - 1) / per);
  const int kt = sw_kt(k), bm = sw_bm(kt);
  dim3 grid((unsigned)((rows_out + bm - 1) / bm), (k + kt - 1) / kt, splits);
  float* p = splits > 1 ? (float*)part : nullptr;
  // whole-vector loads need every row start and the base 16-byte (float) /
  // 8-byte (16-bit) aligned
  const size_t xa = sizeof(TX) * 4;
  const bool vec = (ldx * (int64_t)sizeof(TX)) % (int64_t)xa == 0 && ((uintptr_t)X % xa) == 0 &&
                   (ldb % 4) == 0 && ((uintptr_t)B % 16) == 0;
  note_launch(splits > 1 ? 2 : 1);
#define SW32(V, K)                                                                         \
  sweep32_kernel<TX, TRANS, V, K><<<grid, SW_T, 0, s>>>((const TX*)X, m, n, ldx, (const float*)B, \
                                                        ldb, k, (float*)C, ldc, per, p)
  if (kt == 32) {
    if (vec) SW32(true, 32);
    else SW32(false, 32);
  } else {
    if (vec) SW32(true, 64);
    else SW32(false, 64);
  }
#undef SW32
  if (splits > 1) {
    const int64_t total = rows_out * k;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    splitk_reduce<float><<<blocks, 256, 0, s>>>((const float*)part, splits, rows_out, k, (float*)C, ldc);
  }
}

template <bool TRANS>
static void sweep_dispatch(const void* X, int xdt, int64_t m, int64_t n, int64_t ldx, const void* B,
                           int ldb, int k, void* C, int ldc, int fdt, void* part, int num_sms,
                           cudaStream_t s) {
  if (fdt == T_F64) {
    if (xdt == T_F64) sweep_launch<double, double, TRANS>(X, m, n, ldx, B, ldb, k, C, ldc, part, num_sms, s);
    else if (xdt == T_F32) sweep_launch<float, double, TRANS>(X, m, n, ldx, B, ldb, k, C, ldc, part, num_sms, s);
    else if (xdt == T_BF16) sweep_launch<__nv_bfloat16, double, TRANS>(X, m, n, ldx, B, ldb, k, C, ldc, part, num_sms, s);
    else sweep_launch<__half, double, TRANS>(X, m, n, ldx, B, ldb, k, C, ldc, part, num_sms, s);
  } else {
    if (xdt == T_F32) sweep32_launch<float, TRANS>(X, m, n, ldx, B, ldb, k, C, ldc, part, num_sms, s);
    else if (xdt == T_F64) sweep_launch<double, float, TRANS>(X, m, n, ldx, B, ldb, k, C, ldc, part, num_sms, s);
    else if (xdt == T_BF16) sweep32_launch<__nv_bfloat16, TRANS>(X, m, n, ldx, B, ldb, k, C, ldc, part, num_sms, s);
    else sweep32_launch<__half, TRANS>(X, m, n, ldx, B, ldb, k, C, ldc, part, num_sms, s);
  }
}

void launch_xv(const void* X, int xdt, int64_t m, int64_t n, int64_t ldx, const void* B, int ldb,
               int k, void* C, int ldc, int fdt, void* part, int num_sms, cudaStream_t s) {
  if (xdt == T_CSR) {
    launch_spmm(*(const CsrX*)X, false, B, ldb, k, C, ldc, fdt, num_sms, s);
    return;
  }
  sweep_dispatch<false>(X, xdt, m, n, ldx, B, ldb, k, C, ldc, fdt, part, num_sms, s);
}
void launch_xtu(const void* X, int xdt, int64_t m, int64_t n, int64_t ldx, const void* B, int ldb,
                int k, void* C, int ldc, int fdt, void* part, int num_sms, cudaStream_t s) {
  if (xdt == T_CSR) {
    launch_spmm(*(const CsrX*)X, true, B, ldb, k, C, ldc, fdt, num_sms, s);
    return;
  }
  sweep_dispatch<true>(X, xdt, m, n, ldx, B, ldb, k, C, ldc, fdt, part, num_sms, s);
}

// ------------------------------------------------------------------- Grams
// Partial A^T B over a contiguous row chunk per block; NPART blocks.
constexpr int GRAM_T = 256;
constexpr int GRAM_ROWS = 32;
constexpr int GRAM_PER_T = (LMAX * LMAX + GRAM_T - 1) / GRAM_T;

// Within a block the products are summed in the factor type TF (FP64 for the
// plain form; FP32 for the FP32 form, whose factors carry FP32 precision
// anyway); the NPART block partials are then summed in FP64.
template <typename TF>
__global__ void __launch_bounds__(GRAM_T)
gram_partial(const TF* __restrict__ A, int lda, int ka, const TF* __restrict__ B, int ldb, int kb,
             int64_t rows, double* __restrict__ part) {
  __shared__ TF As[GRAM_ROWS][LMAX];
  __shared__ TF Bs[GRAM_ROWS][LMAX];
  const int64_t chunk = (rows + NPART - 1) / NPART;
  const int64_t r0 = (int64_t)blockIdx.x * chunk;
  const int64_t r1 = min(rows, r0 + chunk);
  const int nk = ka * kb;
  TF acc[GRAM_PER_T];
#pragma unroll
  for (int q = 0; q < GRAM_PER_T; ++q) acc[q] = TF(0);
  for (int64_t t0 = r0; t0 < r1; t0 += GRAM_ROWS) {
    int nr = (int)min((int64_t)GRAM_ROWS, r1 - t0);
    for (int e = threadIdx.x; e < GRAM_ROWS * ka; e += GRAM_T) {
      int rr = e / ka, cc = e % ka;
      As[rr][cc] = rr < nr ? A[(t0 + rr) * lda + cc] : TF(0);
    }
    for (int e = threadIdx.x; e < GRAM_ROWS * kb; e += GRAM_T) {
      int rr = e / kb, cc = e % kb;
      Bs[rr][cc] = rr < nr ? B[(t0 + rr) * ldb + cc] : TF(0);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < GRAM_PER_T; ++q) {
      int e = threadIdx.x + q * GRAM_T;
      if (e < nk) {
        int i = e / kb, j = e % kb;
        TF s = acc[q];
        for (int rr = 0; rr < nr; ++rr) s = fma(As[rr][i], Bs[rr][j], s);
        acc[q] = s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < GRAM_PER_T; ++q) {
    int e = threadIdx.x + q * GRAM_T;
    if (e < nk) part[(int64_t)blockIdx.x * nk + e] = (double)acc[q];
  }
}

// Eight interleaved accumulators (partial b goes to accumulator b % 8), then a
// fixed pairwise combine: the order is fixed, so the sum is reproducible, and
// the eight independent chains hide the load latency.
// Fixed-order sum of the NPART block partials of each of `width` entries:
// block b takes entries 32 b .. 32 b + 31 (one per lane), warp w sums
// partials 32 w .. 32 w + 31 of its lane's entry in four chains, and the
// eight warp sums are added in a fixed tree.
static_assert(NPART == 256, "part_reduce: eight warps of 32 partials");
__global__ void __launch_bounds__(256)
part_reduce(const double* __restrict__ part, int width, double* __restrict__ out) {
  __shared__ double ws[8][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + lane;
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  if (e < width) {
    const double* p = part + (int64_t)(w * 32) * width + e;
#pragma unroll
    for (int b = 0; b < 32; b += 4)
#pragma unroll
      for (int q = 0; q < 4; ++q) a[q] += __ldcg(p + (int64_t)(b + q) * width);
  }
  ws[w][lane] = (a[0] + a[1]) + (a[2] + a[3]);
  __syncthreads();
  if (w == 0 && e < width)
    out[e] = ((ws[0][lane] + ws[1][lane]) + (ws[2][lane] + ws[3][lane])) +
             ((ws[4][lane] + ws[5][lane]) + (ws[6][lane] + ws[7][lane]));
}

static void part_reduce_launch(const double* part, int width, double* out, cudaStream_t s) {
  part_reduce<<<(width + 31) / 32, 256, 0, s>>>(part, width, out);
}

void launch_part_reduce(const double* part, int width, double* out, cudaStream_t s) {
  note_launch(1);
  part_reduce_launch(part, width, out, s);
}

void launch_gram(const void* A, int lda, int ka, const void* B, int ldb, int kb, int64_t rows,
                 int fdt, double* part, double* G, cudaStream_t s) {
  note_launch(2);
  if (fdt == T_F64)
    gram_partial<double><<<NPART, GRAM_T, 0, s>>>((const double*)A, lda, ka, (const double*)B, ldb, kb, rows, part);
  else
    gram_partial<float><<<NPART, GRAM_T, 0, s>>>((const float*)A, lda, ka, (const float*)B, ldb, kb, rows, part);
  int w = ka * kb;
  part_reduce_launch(part, w, G, s);
}

// ------------------------------------------------------------ dot product
template <typename TF>
__global__ void __launch_bounds__(256)
dot_partial(const TF* __restrict__ A, int lda, const TF* __restrict__ B, int ldb, int k,
            int64_t rows, double* __restrict__ part) {
  __shared__ double sh[256];
  const int64_t chunk = (rows + NPART - 1) / NPART;
  const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(rows, r0 + chunk);
  double s = 0.0;
  const int64_t total = (r1 > r0 ? r1 - r0 : 0) * k;
  for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
    int64_t i = r0 + e / k;
    int j = (int)(e % k);
    s = fma((double)A[i * lda + j], (double)B[i * ldb + j], s);
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

void launch_dot(const void* A, int lda, const void* B, int ldb, int k, int64_t rows, int fdt,
                double* part, double* out, cudaStream_t s) {
  note_launch(2);
  if (fdt == T_F64)
    dot_partial<double><<<NPART, 256, 0, s>>>((const double*)A, lda, (const double*)B, ldb, k, rows, part);
  else
    dot_partial<float><<<NPART, 256, 0, s>>>((const float*)A, lda, (const float*)B, ldb, k, rows, part);
  part_reduce_launch(part, 1, out, s);
}

// ---------------------------------------------------------------- ||X||^2
// Each block sums the squares of a chunk of rows; the domain check (x >= 0,
// finite) rides along.  FP64 X: FP64 squares and sums.  FP32 and 16-bit X
// (exact in FP32): the checks in FP32 and each thread's sum kept as an
// unevaluated FP32 pair -- x^2 split exactly by one FMA, added by Knuth's
// two-sum -- so the FP64 pipe (a small fraction of the FP32 rate on this
// GPU) only sees the final pair; eight such pairs (rows i mod 8) per thread.
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }

__device__ __forceinline__ void two_sum_sq(float x, float& hi, float& lo) {
  const float p = __fmul_rn(x, x);
  const float pe = fmaf(x, x, -p);
  const float sm = __fadd_rn(hi, p);
  const float bv = __fsub_rn(sm, hi);
  const float er = __fadd_rn(__fsub_rn(hi, __fsub_rn(sm, bv)), __fsub_rn(p, bv));
  hi = sm;
  lo = __fadd_rn(lo, __fadd_rn(er, pe));
}

template <typename TX>
__global__ void __launch_bounds__(256)
normx2_partial(const TX* __restrict__ X, int64_t m, int64_t n, int64_t ldx,
               double* __restrict__ part, int* err) {
  __shared__ double sh[256];
  const int64_t chunk = (m + NPART - 1) / NPART;
  const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(m, r0 + chunk);
  int bad = 0;
  double s;
  if constexpr (sizeof(TX) == 8) {
    double s8[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) s8[u] = 0.0;
    for (int64_t i = r0; i < r1; i += 8)
      for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        double x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = i + u < r1 ? to_d(X[(i + u) * ldx + j]) : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (!(x[u] >= 0.0) || isinf(x[u])) bad = 1;
          s8[u] = fma(x[u], x[u], s8[u]);
        }
      }
    s = ((s8[0] + s8[1]) + (s8[2] + s8[3])) + ((s8[4] + s8[5]) + (s8[6] + s8[7]));
  } else {
    float hi[8], lo[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) hi[u] = lo[u] = 0.f;
    for (int64_t i = r0; i < r1; i += 8)
      for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        float x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = i + u < r1 ? to_f(X[(i + u) * ldx + j]) : 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (!(x[u] >= 0.f) || isinf(x[u])) bad = 1;
          two_sum_sq(x[u], hi[u], lo[u]);
        }
      }
    double d8[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) d8[u] = (double)hi[u] + (double)lo[u];
    s = ((d8[0] + d8[1]) + (d8[2] + d8[3])) + ((d8[4] + d8[5]) + (d8[6] + d8[7]));
  }
  if (bad) atomicOr(err, ERR_DOMAIN);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// FP32 X with 16-byte aligned rows: the same sums, each thread reading four
// adjacent entries of eight rows per step (128 bytes in flight per thread
// instead of 32; the scalar form left the pass latency-bound at about a
// seventh of the memory bandwidth).  The four entries go into the row's pair
// in column order.
__device__ __forceinline__ void sq4(const float4 v, float& hi, float& lo, int& bad) {
  const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if (!(e[c] >= 0.f) || isinf(e[c])) bad = 1;
    two_sum_sq(e[c], hi, lo);
  }
}

__global__ void __launch_bounds__(256)
normx2_partial_f4(const float* __restrict__ X, int64_t m, int64_t n, int64_t ldx,
                  double* __restrict__ part, int* err) {
  __shared__ double sh[256];
  const int64_t chunk = (m + NPART - 1) / NPART;
  const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(m, r0 + chunk);
  const int64_t n4 = n / 4;
  int bad = 0;
  float hi[8], lo[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) hi[u] = lo[u] = 0.f;
  for (int64_t i = r0; i < r1; i += 8) {
    for (int64_t j4 = threadIdx.x; j4 < n4; j4 += blockDim.x) {
      float4 x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        x[u] = i + u < r1 ? __ldg(reinterpret_cast<const float4*>(X + (i + u) * ldx) + j4)
                          : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 8; ++u) sq4(x[u], hi[u], lo[u], bad);
    }
    for (int64_t j = 4 * n4 + threadIdx.x; j < n; j += blockDim.x) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float x = i + u < r1 ? X[(i + u) * ldx + j] : 0.f;
        if (!(x >= 0.f) || isinf(x)) bad = 1;
        two_sum_sq(x, hi[u], lo[u]);
      }
    }
  }
  double d8[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) d8[u] = (double)hi[u] + (double)lo[u];
  double sum = ((d8[0] + d8[1]) + (d8[2] + d8[3])) + ((d8[4] + d8[5]) + (d8[6] + d8[7]));
  if (bad) atomicOr(err, ERR_DOMAIN);
  sum = block_sum(sum, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = sum;
}

void launch_normx2(const void* X, int xdt, int64_t m, int64_t n, int64_t ldx, double* part,
                   double* out, int* err, cudaStream_t s) {
  if (xdt == T_CSR) {
    launch_csr_normx2(*(const CsrX*)X, part, out, err, s);
    return;
  }
  note_launch(2);
  if (xdt == T_F64) normx2_partial<double><<<NPART, 256, 0, s>>>((const double*)X, m, n, ldx, part, err);
  else if (xdt == T_F32 && ldx % 4 == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0)
    normx2_partial_f4<<<NPART, 256, 0, s>>>((const float*)X, m, n, ldx, part, err);
  else if (xdt == T_F32) normx2_partial<float><<<NPART, 256, 0, s>>>((const float*)X, m, n, ldx, part, err);
  else if (xdt == T_BF16) normx2_partial<__nv_bfloat16><<<NPART, 256, 0, s>>>((const __nv_bfloat16*)X, m, n, ldx, part, err);
  else normx2_partial<__half><<<NPART, 256, 0, s>>>((const __half*)X, m, n, ldx, part, err);
  part_reduce_launch(part, 1, out, s);
}

// ------------------------------------------------------- direct residual
// Each block owns a chunk of rows; per 16-row x 128-column tile it stages U
// and V rows in shared memory and forms x_ij - u_i . v_j for every entry.
constexpr int RD_ROWS = 16, RD_COLS = 64;

template <typename TX, typename TF>
__global__ void __launch_bounds__(RD_COLS)
residual_partial(const TX* __restrict__ X, int64_t m, int64_t n, int64_t ldx,
                 const TF* __restrict__ U, const TF* __restrict__ V, int r,
                 double* __restrict__ part) {
  __shared__ TF Us[RD_ROWS][RMAX];
  __shared__ TF Vs[RMAX][RD_COLS + 1];
  __shared__ double sh[RD_COLS];
  const int64_t chunk = (m + NPART - 1) / NPART;
  const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(m, r0 + chunk);
  double s = 0.0;
  for (int64_t i0 = r0; i0 < r1; i0 += RD_ROWS) {
    int nr = (int)min((int64_t)RD_ROWS, r1 - i0);
    __syncthreads();
    for (int e = threadIdx.x; e < RD_ROWS * r; e += RD_COLS) {
      int rr = e / r, cc = e % r;
      Us[rr][cc] = rr < nr ? U[(i0 + rr) * r + cc] : TF(0);
    }
    for (int64_t j0 = 0; j0 < n; j0 += RD_COLS) {
      int nc = (int)min((int64_t)RD_COLS, n - j0);
      __syncthreads();
      for (int e = threadIdx.x; e < RD_COLS * r; e += RD_COLS) {
        int jj = e / r, cc = e % r;
        Vs[cc][jj] = jj < nc ? V[(j0 + jj) * r + cc] : TF(0);
      }
      __syncthreads();
      int jj = threadIdx.x;
      if (jj < nc) {
        for (int rr = 0; rr < nr; ++rr) {
          TF dotv = TF(0);
          for (int c = 0; c < r; ++c) dotv = fma(Us[rr][c], Vs[c][jj], dotv);
          double e = to_d(X[(i0 + rr) * ldx + j0 + jj]) - (double)dotv;
          s = fma(e, e, s);
        }
      }
    }
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// The same for FP32 factors (FP32 or 16-bit X): the u . v dots in FP32 as
// above, register-tiled.  A CTA keeps a 128-row tile of U in shared memory
// (U^T, r rows) and walks 64-column tiles of V; thread (tr, tc) of 16 x 16
// owns entries (tr + 16 i, tc + 16 j), i < 8, j < 4, and requests its X
// entries before forming the dots.  Each entry's x - u . v is formed exactly
// (as an FP32 pair: the value the FP64 difference gives) and its square
// summed in an FP32 pair per thread to about 2^-48, so the FP64 pipe only
// sees the pair totals; NPART partials.
constexpr int RS_BM = 128, RS_BN = 64, RS_T = 256, RS_GY = NPART / 64;

template <typename TX>
__global__ void __launch_bounds__(RS_T)
residual32_partial(const TX* __restrict__ X, int64_t m, int64_t n, int64_t ldx,
                   const float* __restrict__ U, const float* __restrict__ V, int r,
                   double* __restrict__ part) {
  extern __shared__ __align__(16) float rsm[];
  float* Ut = rsm;                         // r x (RS_BM + 1): Ut[c * (RS_BM + 1) + i]
  float* Vt = Ut + r * (RS_BM + 1);        // r x (RS_BN + 1)
  __shared__ double sh[RS_T];
  const int t = threadIdx.x, tr = t / 16, tc = t % 16;
  const int64_t ntile_r = (m + RS_BM - 1) / RS_BM, ntile_c = (n + RS_BN - 1) / RS_BN;
  float hi = 0.f, lo = 0.f;
  for (int64_t ti = blockIdx.x; ti < ntile_r; ti += gridDim.x) {
    const int64_t row0 = ti * RS_BM;
    __syncthreads();
    for (int e = t; e < RS_BM * r; e += RS_T) {
      const int i = e / r, c = e % r;
      Ut[c * (RS_BM + 1) + i] = row0 + i < m ? U[(row0 + i) * r + c] : 0.f;
    }
    for (int64_t tj = blockIdx.y; tj < ntile_c; tj += gridDim.y) {
      const int64_t col0 = tj * RS_BN;
      float x[8][4];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int64_t gr = row0 + tr + 16 * i, gc = col0 + tc + 16 * j;
          x[i][j] = (gr < m && gc < n) ? ld1(X + gr * ldx + gc) : 0.f;
        }
      __syncthreads();   // the previous tile's dots are done with Vt
      for (int e = t; e < RS_BN * r; e += RS_T) {
        const int jj = e / r, c = e % r;
        Vt[c * (RS_BN + 1) + jj] = col0 + jj < n ? V[(col0 + jj) * r + c] : 0.f;
      }
      __syncthreads();
      float d[8][4];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) d[i][j] = 0.f;
      for (int c = 0; c < r; ++c) {
        float a[8], b[4];
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = Ut[c * (RS_BM + 1) + tr + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Vt[c * (RS_BN + 1) + tc + 16 * j];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) d[i][j] = fmaf(a[i], b[j], d[i][j]);
      }
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          // e = x - d exactly as eh + el (two-difference), then e^2 = p + pe
          // + 2 eh el (+ el^2, below 2^-48 of e^2) into the pair (hi, lo);
          // zero outside the matrix (both terms zero)
          const float xv = x[i][j], nd = -d[i][j];
          const float eh = __fadd_rn(xv, nd);
          const float bv = __fsub_rn(eh, xv);
          const float el = __fadd_rn(__fsub_rn(xv, __fsub_rn(eh, bv)), __fsub_rn(nd, bv));
          const float p = __fmul_rn(eh, eh);
          const float pe = fmaf(eh, eh, -p);
          const float sm = __fadd_rn(hi, p);
          const float bw = __fsub_rn(sm, hi);
          const float er = __fadd_rn(__fsub_rn(hi, __fsub_rn(sm, bw)), __fsub_rn(p, bw));
          hi = sm;
          lo = __fadd_rn(lo, __fadd_rn(er, __fadd_rn(pe, __fmul_rn(2.f * eh, el))));
        }
    }
  }
  double s = (double)hi + (double)lo;
  s = block_sum(s, sh);
  if (t == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = s;
}

template <typename TX>
static void residual32_launch(const void* X, int64_t m, int64_t n, int64_t ldx, const void* U,
                              const void* V, int r, double* part, cudaStream_t s) {
  const size_t smem = sizeof(float) * ((size_t)r * (RS_BM + 1) + (size_t)r * (RS_BN + 1));
  cudaFuncSetAttribute(residual32_partial<TX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  residual32_partial<TX><<<dim3(NPART / RS_GY, RS_GY), RS_T, smem, s>>>(
      (const TX*)X, m, n, ldx, (const float*)U, (const float*)V, r, part);
}

void launch_residual_direct(const void* X, int xdt, int64_t m, int64_t n, int64_t ldx,
                            const void* U, const void* V, int r, int fdt, double* part,
                            double* out, cudaStream_t s) {
  note_launch(2);
#define RD_LAUNCH(TX, TF) \
  residual_partial<TX, TF><<<NPART, RD_COLS, 0, s>>>((const TX*)X, m, n, ldx, (const TF*)U, (const TF*)V, r, part)
  if (fdt == T_F64) {
    if (xdt == T_F64) RD_LAUNCH(double, double);
    else if (xdt == T_F32) RD_LAUNCH(float, double);
    else if (xdt == T_BF16) RD_LAUNCH(__nv_bfloat16, double);
    else RD_LAUNCH(__half, double);
  } else {
    if (xdt == T_F64) RD_LAUNCH(double, float);
    else if (xdt == T_F32) residual32_launch<float>(X, m, n, ldx, U, V, r, part, s);
    else if (xdt == T_BF16) residual32_launch<__nv_bfloat16>(X, m, n, ldx, U, V, r, part, s);
    else residual32_launch<__half>(X, m, n, ldx, U, V, r, part, s);
  }
#undef RD_LAUNCH
  part_reduce_launch(part, 1, out, s);
}

// ------------------------------------------------------------------ Omega
template <typename TF>
__global__ void omega_kernel(TF* F, int64_t rows, int k, uint64_t seed) {
  int64_t total = rows * k;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    F[e] = (TF)hash_uniform(seed, (uint64_t)(e / k), (uint64_t)(e % k));
}

void launch_omega(void* F, int fdt, int64_t rows, int k, uint64_t seed, cudaStream_t s) {
  note_launch(1);
  int64_t total = rows * k;
  int blocks = (int)min((int64_t)4096, (total + 255) / 256);
  if (fdt == T_F64) omega_kernel<double><<<blocks, 256, 0, s>>>((double*)F, rows, k, seed);
  else omega_kernel<float><<<blocks, 256, 0, s>>>((float*)F, rows, k, seed);
}

}  // namespace enmf
