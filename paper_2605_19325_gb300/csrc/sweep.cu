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
    if (xdt == T_F32) sweep_launch<float, float, TRANS>(X, m, n, ldx, B, ldb, k, C, ldc, part, num_sms, s);
    else if (xdt == T_F64) sweep_launch<double, float, TRANS>(X, m, n, ldx, B, ldb, k, C, ldc, part, num_sms, s);
    else if (xdt == T_BF16) sweep_launch<__nv_bfloat16, float, TRANS>(X, m, n, ldx, B, ldb, k, C, ldc, part, num_sms, s);
    else sweep_launch<__half, float, TRANS>(X, m, n, ldx, B, ldb, k, C, ldc, part, num_sms, s);
  }
}

void launch_xv(const void* X, int xdt, int64_t m, int64_t n, int64_t ldx, const void* B, int ldb,
               int k, void* C, int ldc, int fdt, void* part, int num_sms, cudaStream_t s) {
  sweep_dispatch<false>(X, xdt, m, n, ldx, B, ldb, k, C, ldc, fdt, part, num_sms, s);
}
void launch_xtu(const void* X, int xdt, int64_t m, int64_t n, int64_t ldx, const void* B, int ldb,
                int k, void* C, int ldc, int fdt, void* part, int num_sms, cudaStream_t s) {
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
__global__ void part_reduce(const double* __restrict__ part, int width, double* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < width; e += gridDim.x * blockDim.x) {
    double a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll 4
    for (int b = 0; b < NPART; b += 8)
#pragma unroll
      for (int q = 0; q < 8; ++q) a[q] += part[(int64_t)(b + q) * width + e];
    out[e] = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
  }
}

void launch_part_reduce(const double* part, int width, double* out, cudaStream_t s) {
  note_launch(1);
  part_reduce<<<(width + 255) / 256, 256, 0, s>>>(part, width, out);
}

void launch_gram(const void* A, int lda, int ka, const void* B, int ldb, int kb, int64_t rows,
                 int fdt, double* part, double* G, cudaStream_t s) {
  note_launch(2);
  if (fdt == T_F64)
    gram_partial<double><<<NPART, GRAM_T, 0, s>>>((const double*)A, lda, ka, (const double*)B, ldb, kb, rows, part);
  else
    gram_partial<float><<<NPART, GRAM_T, 0, s>>>((const float*)A, lda, ka, (const float*)B, ldb, kb, rows, part);
  int w = ka * kb;
  part_reduce<<<(w + 255) / 256, 256, 0, s>>>(part, w, G);
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
  part_reduce<<<1, 32, 0, s>>>(part, 1, out);
}

// ---------------------------------------------------------------- ||X||^2
template <typename TX>
__global__ void __launch_bounds__(256)
normx2_partial(const TX* __restrict__ X, int64_t m, int64_t n, int64_t ldx,
               double* __restrict__ part, int* err) {
  __shared__ double sh[256];
  const int64_t chunk = (m + NPART - 1) / NPART;
  const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(m, r0 + chunk);
  double s = 0.0;
  int bad = 0;
  for (int64_t i = r0; i < r1; ++i)
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
      double x = to_d(X[i * ldx + j]);
      if (!(x >= 0.0) || isinf(x)) bad = 1;
      s = fma(x, x, s);
    }
  if (bad) atomicOr(err, ERR_DOMAIN);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

void launch_normx2(const void* X, int xdt, int64_t m, int64_t n, int64_t ldx, double* part,
                   double* out, int* err, cudaStream_t s) {
  note_launch(2);
  if (xdt == T_F64) normx2_partial<double><<<NPART, 256, 0, s>>>((const double*)X, m, n, ldx, part, err);
  else if (xdt == T_F32) normx2_partial<float><<<NPART, 256, 0, s>>>((const float*)X, m, n, ldx, part, err);
  else if (xdt == T_BF16) normx2_partial<__nv_bfloat16><<<NPART, 256, 0, s>>>((const __nv_bfloat16*)X, m, n, ldx, part, err);
  else normx2_partial<__half><<<NPART, 256, 0, s>>>((const __half*)X, m, n, ldx, part, err);
  part_reduce<<<1, 32, 0, s>>>(part, 1, out);
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
    else if (xdt == T_F32) RD_LAUNCH(float, float);
    else if (xdt == T_BF16) RD_LAUNCH(__nv_bfloat16, float);
    else RD_LAUNCH(__half, float);
  }
#undef RD_LAUNCH
  part_reduce<<<1, 32, 0, s>>>(part, 1, out);
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
