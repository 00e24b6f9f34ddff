// X given by its stored entries in compressed rows (the sparse form; the
// Reuters experiment of Sec. 5 is a 99.84 % sparse document-term matrix).
// The method is unchanged: only the products X B and X^T B and ||X||^2
// touch X, and each reads the stored entries once.
//
//   * X B   -- one warp per row (lane t owns the columns l = t + 32 e of B
//     and of the output).  The warp walks the row's entries in order, 32 at
//     a time: lane t loads the (column, value) pair of entry p0 + t
//     (coalesced), then every entry's pair is broadcast by a shuffle and the
//     warp reads B's row of that column (coalesced, mostly from L2: B is
//     (m or n) x k).  A whole warp shares one row, so every shuffle runs
//     with all 32 lanes converged.  Four
//     entries' rows of B are requested before the first multiply.  Each
//     output row is summed in entry order, so results are deterministic.
//   * X^T B -- the same kernel on the transpose, which the context builds
//     once per X: a stable counting sort of the entries by column, so every
//     column's entries stay in row order (deterministic, like the rows).
//
// The transpose: rows are cut into B blocks of consecutive rows.  Pass 1
// counts entries per (block, column); pass 2 turns the counts into, per
// column, the number of that column's entries in earlier blocks (and the
// column totals); a scan of the totals gives the column pointers; pass 3
// lets each block walk its rows in order and place every entry at
// col_ptr[c] + (earlier blocks' entries of c) + (its own earlier entries of
// c).  Within one row the columns are distinct, so the threads of a block
// handle a row's entries at once; rows follow one another in order.
#include <vector>

#include "internal.h"

namespace enmf {
namespace {

constexpr int SP_T = 256;

template <typename T>
__device__ __forceinline__ T shfl(T v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}

static inline size_t al256d(size_t b) { return (b + 255) / 256 * 256; }

// ------------------------------------------------------------- checks
// One thread per row: row_ptr[0] = 0, row_ptr nondecreasing, row_ptr[m] = nnz,
// columns in [0, n) strictly increasing within each row (ERR_FORMAT); values
// finite and >= 0 (ERR_DOMAIN).
template <typename TV>
__global__ void __launch_bounds__(SP_T)
csr_check_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                 const TV* __restrict__ val, int64_t m, int64_t n, int64_t nnz, int* err) {
  int bad_fmt = 0, bad_dom = 0;
  for (int64_t i = (int64_t)blockIdx.x * SP_T + threadIdx.x; i < m; i += (int64_t)gridDim.x * SP_T) {
    const int64_t a = rp[i], b = rp[i + 1];
    if ((i == 0 && a != 0) || (i == m - 1 && b != nnz) || a < 0 || b < a || b > nnz) {
      bad_fmt = 1;
      continue;
    }
    int32_t prev = -1;
    for (int64_t p = a; p < b; ++p) {
      const int32_t c = col[p];
      if (c <= prev || (int64_t)c >= n) bad_fmt = 1;
      prev = c;
      const double v = (double)val[p];
      if (!(v >= 0.0) || isinf(v)) bad_dom = 1;
    }
  }
  if (bad_fmt) atomicOr(err, ERR_FORMAT);
  if (bad_dom) atomicOr(err, ERR_DOMAIN);
}

// ------------------------------------------------------------ transpose
__global__ void __launch_bounds__(SP_T)
csr_hist_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ col, int64_t m,
                int64_t n, int64_t rows_per_blk, int* __restrict__ hist) {
  const int64_t b = blockIdx.x;
  const int64_t r0 = b * rows_per_blk, r1 = min(m, r0 + rows_per_blk);
  if (r0 >= r1) return;
  const int64_t p0 = rp[r0], p1 = rp[r1];
  int* h = hist + b * n;
  for (int64_t p = p0 + threadIdx.x; p < p1; p += SP_T) atomicAdd(&h[col[p]], 1);
}

// Per column c: cnt[c] = sum over blocks of hist[b][c]; hist[b][c] becomes
// the entries of c in blocks before b.
__global__ void __launch_bounds__(SP_T)
csr_colsum_kernel(int* __restrict__ hist, int64_t nblk, int64_t n, int64_t* __restrict__ cnt) {
  for (int64_t c = (int64_t)blockIdx.x * SP_T + threadIdx.x; c < n; c += (int64_t)gridDim.x * SP_T) {
    int64_t s = 0;
    for (int64_t b = 0; b < nblk; ++b) {
      const int h = hist[b * n + c];
      hist[b * n + c] = (int)s;
      s += h;
    }
    cnt[c] = s;
  }
}

// Exclusive scan of cnt (n entries) into ptr (n + 1 entries), three passes
// over chunks of SCAN_CHUNK entries.
constexpr int SCAN_CHUNK = 4096;

__global__ void __launch_bounds__(SP_T)
scan_chunk_sums(const int64_t* __restrict__ cnt, int64_t n, int64_t* __restrict__ csum) {
  __shared__ int64_t sh[SP_T];
  const int64_t c0 = (int64_t)blockIdx.x * SCAN_CHUNK;
  int64_t s = 0;
  for (int64_t e = c0 + threadIdx.x; e < min(n, c0 + SCAN_CHUNK); e += SP_T) s += cnt[e];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = SP_T / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) csum[blockIdx.x] = sh[0];
}

// One block: exclusive scan of the nc chunk sums in place (sequential per
// thread over a contiguous run, then a scan of the run totals).
__global__ void __launch_bounds__(SP_T) scan_chunk_offsets(int64_t* __restrict__ csum, int64_t nc) {
  __shared__ int64_t tot[SP_T];
  const int64_t per = (nc + SP_T - 1) / SP_T;
  const int64_t a = threadIdx.x * per, b = min(nc, a + per);
  int64_t s = 0;
  for (int64_t e = a; e < b; ++e) s += csum[e];
  tot[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t run = 0;
    for (int t = 0; t < SP_T; ++t) {
      const int64_t v = tot[t];
      tot[t] = run;
      run += v;
    }
  }
  __syncthreads();
  int64_t run = tot[threadIdx.x];
  for (int64_t e = a; e < b; ++e) {
    const int64_t v = csum[e];
    csum[e] = run;
    run += v;
  }
}

// Block per chunk: the chunk's exclusive prefix, by a block scan of the
// per-thread runs.
__global__ void __launch_bounds__(SP_T)
scan_chunk_apply(const int64_t* __restrict__ cnt, int64_t n, const int64_t* __restrict__ csum,
                 int64_t* __restrict__ ptr) {
  __shared__ int64_t tot[SP_T];
  constexpr int PER = SCAN_CHUNK / SP_T;
  const int64_t c0 = (int64_t)blockIdx.x * SCAN_CHUNK;
  const int64_t a = c0 + (int64_t)threadIdx.x * PER;
  int64_t v[PER];
  int64_t s = 0;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    v[q] = a + q < n ? cnt[a + q] : 0;
    s += v[q];
  }
  tot[threadIdx.x] = s;
  __syncthreads();
  for (int w = 1; w < SP_T; w <<= 1) {   // inclusive Hillis-Steele scan of the run totals
    const int64_t add = (int)threadIdx.x >= w ? tot[threadIdx.x - w] : 0;
    __syncthreads();
    tot[threadIdx.x] += add;
    __syncthreads();
  }
  int64_t run = csum[blockIdx.x] + tot[threadIdx.x] - s;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    if (a + q < n) ptr[a + q] = run;
    run += v[q];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == SP_T - 1) ptr[n] = run;
}

template <typename TV>
__global__ void __launch_bounds__(SP_T)
csr_scatter_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                   const TV* __restrict__ val, int64_t m, int64_t n, int64_t rows_per_blk,
                   const int64_t* __restrict__ col_ptr, int* __restrict__ cur,
                   int32_t* __restrict__ row_t, TV* __restrict__ val_t) {
  const int64_t b = blockIdx.x;
  const int64_t r0 = b * rows_per_blk, r1 = min(m, r0 + rows_per_blk);
  int* cb = cur + b * n;
  for (int64_t i = r0; i < r1; ++i) {
    const int64_t a = rp[i], e = rp[i + 1];
    for (int64_t p = a + threadIdx.x; p < e; p += SP_T) {
      const int32_t c = col[p];
      const int off = cb[c];
      cb[c] = off + 1;   // the row's columns are distinct: no other thread touches cb[c] now
      const int64_t pos = col_ptr[c] + off;
      row_t[pos] = (int32_t)i;
      val_t[pos] = val[p];
    }
    __syncthreads();   // the next row may share columns with this one
  }
}

// ---------------------------------------------------------------- X B
// One warp per work item (at most SPMM_SEG entries of one row): the item's
// entries are read 32 at a time (lane t loads the (column, value) pair of
// entry p0 + t), each pair broadcast by a shuffle; UN entries' rows of B are
// requested before the first multiply.  The next chunk's pairs, and at the
// last chunk the next item's bounds and first pairs, are requested before
// the current chunk is used, so a warp keeps its loads in flight across
// items.  Lane t accumulates the output columns t + 32 e in entry order:
// every item's sum is deterministic.
template <typename TV, typename TF, int E, int UN>
__global__ void __launch_bounds__(SP_T, 6)
spmm_items_kernel(const int32_t* __restrict__ col, const TV* __restrict__ val,
                  const int32_t* __restrict__ item_row, const int64_t* __restrict__ item_p,
                  const int32_t* __restrict__ item_slot, int64_t nitems,
                  const TF* __restrict__ B, int ldb, int k, TF* __restrict__ C, int ldc,
                  TF* __restrict__ part) {
  constexpr int L = 32;
  const int lane = threadIdx.x % L;
  const int64_t g0 = ((int64_t)blockIdx.x * SP_T + threadIdx.x) / L;   // warp-uniform
  const int64_t ng = (int64_t)gridDim.x * SP_T / L;
  if (g0 >= nitems) return;
  // the first item's bounds and pairs
  int64_t a = item_p[2 * g0], b = item_p[2 * g0 + 1];
  int32_t cl = (a + lane < b) ? col[a + lane] : 0;
  TF vl = (a + lane < b) ? (TF)val[a + lane] : TF(0);
  for (int64_t it = g0; it < nitems; it += ng) {
    const int64_t itn = it + ng;
    const int32_t row = item_row[it];
    const int32_t slot = item_slot[it];
    int64_t an = 0, bn = 0;
    if (itn < nitems) {
      an = item_p[2 * itn];
      bn = item_p[2 * itn + 1];
    }
    TF acc[E];
#pragma unroll
    for (int e = 0; e < E; ++e) acc[e] = TF(0);
    int64_t p0 = a;
    while (true) {
      const int cnt = (int)min((int64_t)L, b - p0);
      // the pairs used next: this item's next chunk, else the next item's first
      const bool more = p0 + L < b;
      const int64_t pn = (more ? p0 + L : an) + lane;
      const int64_t en = more ? b : bn;
      const int32_t cn = pn < en ? col[pn] : 0;
      const TF vn = pn < en ? (TF)val[pn] : TF(0);
      for (int j0 = 0; j0 < cnt; j0 += UN) {
        TF bv[UN][E], vv[UN];
#pragma unroll
        for (int u = 0; u < UN; ++u) {
          const int j = j0 + u;
          const int jj = j < cnt ? j : 0;
          const int32_t c = __shfl_sync(0xffffffffu, cl, jj);
          const TF vj = __shfl_sync(0xffffffffu, vl, jj);
          vv[u] = j < cnt ? vj : TF(0);
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int l = lane + L * e;
            bv[u][e] = (j < cnt && l < k) ? B[(int64_t)c * ldb + l] : TF(0);
          }
        }
#pragma unroll
        for (int u = 0; u < UN; ++u)
#pragma unroll
          for (int e = 0; e < E; ++e) acc[e] = fma(vv[u], bv[u][e], acc[e]);
      }
      cl = cn;
      vl = vn;
      if (!more) break;
      p0 += L;
    }
    TF* dst = slot < 0 ? C + (int64_t)row * ldc : part + (int64_t)slot * LMAX;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int l = lane + L * e;
      if (l < k) dst[l] = acc[e];
    }
    a = an;
    b = bn;
  }
}

// The rows cut into several items: their partial rows summed in slot order.
template <typename TF>
__global__ void __launch_bounds__(SP_T)
spmm_fixup_kernel(const int32_t* __restrict__ split_row, const int32_t* __restrict__ split_base,
                  const int32_t* __restrict__ split_cnt, int64_t nsplit,
                  const TF* __restrict__ part, int k, TF* __restrict__ C, int ldc) {
  const int lane = threadIdx.x % 32;
  const int64_t g0 = ((int64_t)blockIdx.x * SP_T + threadIdx.x) / 32;
  const int64_t ng = (int64_t)gridDim.x * SP_T / 32;
  for (int64_t q = g0; q < nsplit; q += ng) {
    const int64_t base = split_base[q];
    const int cnt = split_cnt[q];
    for (int l = lane; l < k; l += 32) {
      TF s = TF(0);
      for (int j = 0; j < cnt; ++j) s += part[(base + j) * LMAX + l];
      C[(int64_t)split_row[q] * ldc + l] = s;
    }
  }
}

// ||X||^2 block partials from the stored values (FP64 sums; every stored
// value must be finite and >= 0, else ERR_DOMAIN).
template <typename TV>
__global__ void __launch_bounds__(SP_T)
csr_sumsq_partial(const TV* __restrict__ val, int64_t nnz, double* __restrict__ part, int* err) {
  __shared__ double sh[SP_T];
  const int64_t chunk = (nnz + NPART - 1) / NPART;
  const int64_t a = (int64_t)blockIdx.x * chunk, b = min(nnz, a + chunk);
  double s = 0.0;
  int bad = 0;
  for (int64_t p = a + threadIdx.x; p < b; p += SP_T) {
    const double v = (double)val[p];
    if (!(v >= 0.0) || isinf(v)) bad = 1;
    s = fma(v, v, s);
  }
  if (bad) atomicOr(err, ERR_DOMAIN);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = SP_T / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

template <typename TV, typename TF>
void spmm_launch(const int32_t* col, const void* val, const SpmmPlan& pl,
                 const void* B, int ldb, int k, void* C, int ldc, int num_sms, cudaStream_t s) {
  const TV* v = (const TV*)val;
  const TF* Bf = (const TF*)B;
  TF* Cf = (TF*)C;
  TF* part = (TF*)pl.partial;
  const int64_t warps_per_blk = SP_T / 32;
  int64_t grid = (pl.nitems + warps_per_blk - 1) / warps_per_blk;
  const int64_t cap = (int64_t)num_sms * 6;   // all resident (at most 42 registers)
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
#define SPK(E, UN)                                                                              \
  spmm_items_kernel<TV, TF, E, UN><<<(int)grid, SP_T, 0, s>>>(                                   \
      col, v, pl.item_row, pl.item_p, pl.item_slot, pl.nitems, Bf, ldb, k, Cf, ldc, part)
  // (measured on the Reuters-sized matrix, r = 40: resident warps matter more
  // than entries per round; 4 per round at 6 blocks per SM beat 8 or 16 at 2-4)
  if (k <= 32) SPK(1, 4);
  else if (k <= 64) SPK(2, 4);
  else SPK(3, 4);
#undef SPK
  if (pl.nsplit > 0) {
    int64_t g2 = (pl.nsplit + warps_per_blk - 1) / warps_per_blk;
    if (g2 > cap) g2 = cap;
    spmm_fixup_kernel<TF><<<(int)g2, SP_T, 0, s>>>(pl.split_row, pl.split_base, pl.split_cnt,
                                                    pl.nsplit, part, k, Cf, ldc);
  }
}

}  // namespace

void launch_csr_check(const CsrX& x, int* err, cudaStream_t s) {
  note_launch(1);
  int64_t grid = (x.m + SP_T - 1) / SP_T;
  if (grid > 4096) grid = 4096;
  if (x.vdt == T_F64)
    csr_check_kernel<double><<<(int)grid, SP_T, 0, s>>>(x.row_ptr, x.col, (const double*)x.val, x.m,
                                                         x.n, x.nnz, err);
  else
    csr_check_kernel<float><<<(int)grid, SP_T, 0, s>>>(x.row_ptr, x.col, (const float*)x.val, x.m,
                                                        x.n, x.nnz, err);
}

size_t csr_transpose_scratch(int64_t m, int64_t n, int64_t* nblk_out, int64_t* rows_per_blk_out) {
  // per-(block, column) counters are kept under 64 Mi ints (256 MB)
  int64_t nblk = (int64_t)(64ll << 20) / (n > 0 ? n : 1);
  if (nblk > 1024) nblk = 1024;
  if (nblk < 1) nblk = 1;
  if (nblk > m) nblk = m;
  const int64_t rpb = (m + nblk - 1) / nblk;
  nblk = (m + rpb - 1) / rpb;
  if (nblk_out) *nblk_out = nblk;
  if (rows_per_blk_out) *rows_per_blk_out = rpb;
  const int64_t nc = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
  return al256d((size_t)nblk * n * sizeof(int)) + al256d((size_t)n * 8) + al256d((size_t)nc * 8);
}

void launch_csr_transpose(const CsrX& x, void* scratch, int64_t* col_ptr, int32_t* row_t,
                          void* val_t, cudaStream_t s) {
  note_launch(6);
  int64_t nblk = 1, rpb = 1;
  csr_transpose_scratch(x.m, x.n, &nblk, &rpb);
  char* w = (char*)scratch;
  int* hist = (int*)w;
  w += al256d((size_t)nblk * x.n * sizeof(int));
  int64_t* cnt = (int64_t*)w;
  w += al256d((size_t)x.n * 8);
  int64_t* csum = (int64_t*)w;
  const int64_t nc = (x.n + SCAN_CHUNK - 1) / SCAN_CHUNK;
  cudaMemsetAsync(hist, 0, (size_t)nblk * x.n * sizeof(int), s);
  csr_hist_kernel<<<(int)nblk, SP_T, 0, s>>>(x.row_ptr, x.col, x.m, x.n, rpb, hist);
  int64_t g = (x.n + SP_T - 1) / SP_T;
  if (g > 4096) g = 4096;
  csr_colsum_kernel<<<(int)g, SP_T, 0, s>>>(hist, nblk, x.n, cnt);
  scan_chunk_sums<<<(int)nc, SP_T, 0, s>>>(cnt, x.n, csum);
  scan_chunk_offsets<<<1, SP_T, 0, s>>>(csum, nc);
  scan_chunk_apply<<<(int)nc, SP_T, 0, s>>>(cnt, x.n, csum, col_ptr);
  if (x.vdt == T_F64)
    csr_scatter_kernel<double><<<(int)nblk, SP_T, 0, s>>>(x.row_ptr, x.col, (const double*)x.val, x.m,
                                                           x.n, rpb, col_ptr, hist, row_t,
                                                           (double*)val_t);
  else
    csr_scatter_kernel<float><<<(int)nblk, SP_T, 0, s>>>(x.row_ptr, x.col, (const float*)x.val, x.m,
                                                          x.n, rpb, col_ptr, hist, row_t,
                                                          (float*)val_t);
}

void launch_spmm(const CsrX& x, bool trans, const void* B, int ldb, int k, void* C, int ldc,
                 int fdt, int num_sms, cudaStream_t s) {
  note_launch(1);
  const int64_t* rp = trans ? x.col_ptr : x.row_ptr;
  const int32_t* ix = trans ? x.row_t : x.col;
  const void* v = trans ? x.val_t : x.val;
  const SpmmPlan& pl = x.plan[trans ? 1 : 0];
  if (pl.nsplit > 0) note_launch(1);
  (void)rp;
  if (fdt == T_F64) spmm_launch<double, double>(ix, v, pl, B, ldb, k, C, ldc, num_sms, s);
  else spmm_launch<float, float>(ix, v, pl, B, ldb, k, C, ldc, num_sms, s);
}

// The items of one product from its row pointers (host copy `rp`, rows + 1
// entries), written to the plan's device arrays (synchronous copies on s).
bool build_spmm_plan(const int64_t* rp, int64_t rows, SpmmPlan& pl, cudaStream_t s) {
  std::vector<int32_t> irow, islot, srow, sbase, scnt;
  std::vector<int64_t> ip;
  irow.reserve((size_t)rows + 16);
  int32_t slot = 0;
  for (int64_t i = 0; i < rows; ++i) {
    const int64_t len = rp[i + 1] - rp[i];
    const int64_t nseg = len > SPMM_SEG ? (len + SPMM_SEG - 1) / SPMM_SEG : 1;
    if (nseg > 1) {
      srow.push_back((int32_t)i);
      sbase.push_back(slot);
      scnt.push_back((int32_t)nseg);
    }
    for (int64_t g = 0; g < nseg; ++g) {
      irow.push_back((int32_t)i);
      const int64_t a = rp[i] + g * SPMM_SEG;
      ip.push_back(a);
      ip.push_back(a + SPMM_SEG < rp[i + 1] ? a + SPMM_SEG : rp[i + 1]);
      islot.push_back(nseg > 1 ? slot++ : -1);
    }
  }
  pl.nitems = (int64_t)irow.size();
  pl.nsplit = (int64_t)srow.size();
  bool ok = true;
  auto put = [&](int32_t* dst, const std::vector<int32_t>& v) {
    if (!v.empty() && cudaMemcpyAsync(dst, v.data(), v.size() * 4, cudaMemcpyHostToDevice, s) !=
                          cudaSuccess)
      ok = false;
  };
  put(pl.item_row, irow);
  put(pl.item_slot, islot);
  if (!ip.empty() && cudaMemcpyAsync(pl.item_p, ip.data(), ip.size() * 8, cudaMemcpyHostToDevice,
                                     s) != cudaSuccess)
    ok = false;
  put(pl.split_row, srow);
  put(pl.split_base, sbase);
  put(pl.split_cnt, scnt);
  if (cudaStreamSynchronize(s) != cudaSuccess) ok = false;
  return ok;
}

void launch_csr_normx2(const CsrX& x, double* part, double* out, int* err, cudaStream_t s) {
  note_launch(2);
  if (x.vdt == T_F64)
    csr_sumsq_partial<double><<<NPART, SP_T, 0, s>>>((const double*)x.val, x.nnz, part, err);
  else
    csr_sumsq_partial<float><<<NPART, SP_T, 0, s>>>((const float*)x.val, x.nnz, part, err);
  launch_part_reduce(part, 1, out, s);
}

}  // namespace enmf
