// Matrix completion (App. C, Algorithm eNMC) on the sparse form's pattern:
// the stored entries of X are the KNOWN entries (the mask M_E); the others are
// unknown.  The objective is f^(U, V) = 1/2 ||M_E o (X - U V^T)||_F^2.
//
// With V fixed, row i of U sees only its own known entries:
//   grad_i = (M_E o (U V^T - X)) V row i = u_i G_i - a_i,
//   G_i = sum over the known (i, j) of v_j v_j^T,   a_i = sum x_ij v_j,
// and the exact step of f^ along -g_i (PBCD with M_E, Algorithm 2) is
//   d_i = ||g_i||^2 / sum_j (g_i . v_j)^2 = ||g_i||^2 / (g_i G_i g_i^T).
// So every half step first forms G_i and a_i for all rows from the stored
// entries (nmc_gram_kernel, one pass over the entries and the other factor's
// gathered rows), and the PBCD sweeps then touch only G_i, a_i and the row
// (nmc_pbcd_kernel), with the global stopping test of Algorithm 2 behind a
// grid barrier.  The masked-ALS start solves (G_i + lam c_i I) u_i = a_i per
// row by an FP64 Cholesky factor (nmc_solve_kernel).
//
// Determinism: every sum runs in a fixed order (entries in stored order,
// partials in block order).
#include "internal.h"
#include "lanes.cuh"

namespace enmf {
namespace {

using lanes::FULL;

constexpr int NM_T = 256;   // threads per block; 8 warps

template <typename TF>
__device__ __forceinline__ TF shfl32(TF v, int src) {
  return __shfl_sync(FULL, v, src);
}

template <typename TF>
__device__ __forceinline__ TF warp_sum(TF v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// ------------------------------------------------------------- G_i, a_i
// One block per row (grid-stride).  Entries are taken in chunks of CH: the
// block stages the chunk's rows of B (CH x KP, zero padded) and values, then
// thread t adds, over the chunk in entry order, b_q[l1] b_q[l2] to the entries
// e = t + NM_T s of G_i it owns (l1 = e / KP, l2 = e % KP), and threads
// t < KP add x_q b_q[t] to a_i.
constexpr int CH = 32;

template <typename TV, typename TF, typename TG, int KP>
__global__ void __launch_bounds__(NM_T)
nmc_gram_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ ix,
                const TV* __restrict__ val, int64_t rows, const TF* __restrict__ B, int k,
                TG* __restrict__ G, TG* __restrict__ A) {
  constexpr int OWN = KP * KP / NM_T;   // KP in {16, 32, 48, 64}: 1, 4, 9, 16
  __shared__ TG Bs[CH][KP];
  __shared__ TG xs[CH];
  const int t = threadIdx.x;
  for (int64_t i = blockIdx.x; i < rows; i += gridDim.x) {
    TG acc[OWN];
#pragma unroll
    for (int s = 0; s < OWN; ++s) acc[s] = TG(0);
    TG aacc = TG(0);
    const int64_t p0 = rp[i], p1 = rp[i + 1];
    for (int64_t c0 = p0; c0 < p1; c0 += CH) {
      const int cnt = (int)min((int64_t)CH, p1 - c0);
      __syncthreads();   // the previous chunk has been consumed
      for (int e = t; e < CH * KP; e += NM_T) {
        const int q = e / KP, l = e % KP;
        TG b = TG(0);
        if (q < cnt && l < k) b = (TG)B[(int64_t)ix[c0 + q] * k + l];
        Bs[q][l] = b;
      }
      if (t < CH) xs[t] = t < cnt ? (TG)val[c0 + t] : TG(0);
      __syncthreads();
#pragma unroll
      for (int s = 0; s < OWN; ++s) {
        const int e = t + NM_T * s, l1 = e / KP, l2 = e % KP;
        TG a = acc[s];
        for (int q = 0; q < cnt; ++q) a = fma(Bs[q][l1], Bs[q][l2], a);
        acc[s] = a;
      }
      if (t < KP)
        for (int q = 0; q < cnt; ++q) aacc = fma(xs[q], Bs[q][t], aacc);
    }
    TG* Gi = G + i * (int64_t)KP * KP;
#pragma unroll
    for (int s = 0; s < OWN; ++s) Gi[t + NM_T * s] = acc[s];
    if (t < KP) A[i * KP + t] = aacc;
  }
}

// ------------------------------------------------------------ PBCD rows
// One warp per row; lane t owns the entries l = t + 32 e of u, a, g (E =
// KP / 32 rounded up).  y = w G_i: y_l = sum_m w_m G_i[m][l], w_m from its
// owner lane, G_i's row m read coalesced.
template <typename TF, int KP>
__device__ __forceinline__ void row_times_g(const TF* __restrict__ Gi, const TF (&w)[(KP + 31) / 32],
                                            int k, int lane, TF (&y)[(KP + 31) / 32]) {
  constexpr int E = (KP + 31) / 32;
#pragma unroll
  for (int e = 0; e < E; ++e) y[e] = TF(0);
  for (int mm = 0; mm < k; ++mm) {
    const TF wm = shfl32(w[mm / 32], mm % 32);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int l = lane + 32 * e;
      if (l < KP) y[e] = fma(wm, Gi[mm * KP + l], y[e]);
    }
  }
}

template <typename TF, int KP>
__global__ void __launch_bounds__(NM_T)
nmc_pbcd_kernel(NmcArgs a) {
  constexpr int E = (KP + 31) / 32;
  __shared__ double sh[NM_T];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t w0 = (int64_t)blockIdx.x * (NM_T / 32) + warp;
  const int64_t nw = (int64_t)gridDim.x * (NM_T / 32);
  const int k = a.k;
  TF* F = (TF*)a.F;
  TF* gb = (TF*)a.gbuf;
  const TF* G = (const TF*)a.G;
  const TF* A = (const TF*)a.A;
  DevState* st = a.st;
  const TF sft = (TF)(a.which == 0 ? st->s_u : st->s_v);
  // shift (Eq. 8 / 9), mask, first gradient
  double acc = 0.0;
  for (int64_t i = w0; i < a.rows; i += nw) {
    const TF* Gi = G + i * (int64_t)KP * KP;
    TF u[E], y[E], g[E];
    unsigned long long bits = 0ull;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int l = lane + 32 * e;
      u[e] = l < k ? F[i * k + l] : TF(0);
      if (u[e] < TF(0)) u[e] = u[e] + sft;
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int l = lane + 32 * e;
      const unsigned ok = (l < k && u[e] >= TF(0)) ? 1u : 0u;
      bits |= (unsigned long long)__ballot_sync(FULL, ok) << (32 * e);
    }
    row_times_g<TF, KP>(Gi, u, k, lane, y);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int l = lane + 32 * e;
      const bool on = l < k && ((bits >> l) & 1ull);
      g[e] = on ? y[e] - A[i * KP + l] : TF(0);
      acc = fma((double)g[e], (double)g[e], acc);
      if (l < k) {
        F[i * k + l] = u[e];
        gb[i * k + l] = g[e];
      }
    }
    if (lane == 0) a.mask[i] = bits;
  }
  double bs = lanes::block_sum256(acc, sh);
  if (threadIdx.x == 0) a.part[blockIdx.x] = bs;
  grid_sync(a.bar, a.err);
  double g0 = 0.0;
  {
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += NM_T) s += __ldcg(&a.part[b]);
    g0 = sqrt(lanes::block_sum256(s, sh));
  }
  int iters = 0;
  bool stopped = false;
  for (int it = 0; it < a.pbcd_max_iter && !stopped; ++it) {
    acc = 0.0;
    for (int64_t i = w0; i < a.rows; i += nw) {
      const TF* Gi = G + i * (int64_t)KP * KP;
      const unsigned long long bits = a.mask[i];
      TF u[E], g[E], z[E], y[E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int l = lane + 32 * e;
        u[e] = l < k ? F[i * k + l] : TF(0);
        g[e] = l < k ? gb[i * k + l] : TF(0);
      }
      // d_i = ||g_i||^2 / (g_i G_i g_i^T)   (Eq. 10 with M_E, App. C)
      row_times_g<TF, KP>(Gi, g, k, lane, z);
      TF num = TF(0), den = TF(0);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        num = fma(g[e], g[e], num);
        den = fma(g[e], z[e], den);
      }
      num = warp_sum(num);
      den = warp_sum(den);
      const TF d = (num > TF(0) && den > TF(0)) ? num / den : TF(0);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int l = lane + 32 * e;
        if (l < k && ((bits >> l) & 1ull)) {
          const TF v = u[e] - d * g[e];
          u[e] = v > TF(0) ? v : TF(0);
        }
      }
      row_times_g<TF, KP>(Gi, u, k, lane, y);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int l = lane + 32 * e;
        const bool on = l < k && ((bits >> l) & 1ull);
        g[e] = on ? y[e] - A[i * KP + l] : TF(0);
        acc = fma((double)g[e], (double)g[e], acc);
        if (l < k) {
          F[i * k + l] = u[e];
          gb[i * k + l] = g[e];
        }
      }
    }
    double* pbuf = a.part + (size_t)((it + 1) & 1) * NPART;
    bs = lanes::block_sum256(acc, sh);
    if (threadIdx.x == 0) pbuf[blockIdx.x] = bs;
    grid_sync(a.bar, a.err);
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += NM_T) s += __ldcg(&pbuf[b]);
    const double bc = lanes::block_sum256(s, sh);
    iters = it + 1;
    stopped = sqrt(bc) < a.eps * g0 || bc == 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && a.counts) {
    const int q = a.round;
    if (2 * q + a.which < a.counts_cap) a.counts[2 * q + a.which] = iters;
  }
}

// ------------------------------------------------- masked-ALS row solves
// One warp per row: (G_i + lam c_i I) u_i = a_i with c_i = trace(G_i) / k
// (1 when the trace is 0), by the Cholesky factor L (FP64, in shared memory,
// left-looking by columns), then L y = a, L^T u = y.  G_i and a_i are FP64 in
// every form: a row with fewer known entries than r has a singular G_i, which
// FP32 rounding can push below the tiny ridge.
constexpr int SV_T = 128;   // the solve's threads per block: 4 warps (FP64 factors in shared memory)

template <typename TF, int KP>
__global__ void __launch_bounds__(SV_T)
nmc_solve_kernel(const double* __restrict__ G, const double* __restrict__ A, int64_t rows, int k,
                 double lam, TF* __restrict__ F, int* err) {
  constexpr int LD = KP + 1;
  extern __shared__ double smd[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* L = smd + (size_t)warp * (KP * LD + KP);
  double* y = L + KP * LD;
  const int64_t w0 = (int64_t)blockIdx.x * (SV_T / 32) + warp;
  const int64_t nw = (int64_t)gridDim.x * (SV_T / 32);
  for (int64_t i = w0; i < rows; i += nw) {
    const double* Gi = G + i * (int64_t)KP * KP;
    double tr = 0.0;
    for (int l = lane; l < k; l += 32) tr += (double)Gi[l * KP + l];
    tr = warp_sum(tr);
    const double c = tr > 0.0 ? tr / k : 1.0;
    for (int e = lane; e < k * k; e += 32) {
      const int r0 = e / k, c0 = e % k;
      L[r0 * LD + c0] = (double)Gi[r0 * KP + c0] + (r0 == c0 ? lam * c : 0.0);
    }
    for (int l = lane; l < k; l += 32) y[l] = (double)A[i * KP + l];
    __syncwarp();
    bool ok = true;
    for (int j = 0; j < k; ++j) {
      // L[j][j] = sqrt(A_jj - sum_{p<j} L_jp^2); L[r][j] = (A_rj - sum_p L_rp L_jp) / L_jj
      double dj = L[j * LD + j];
      for (int p = 0; p < j; ++p) dj = fma(-L[j * LD + p], L[j * LD + p], dj);
      if (!(dj > 0.0)) ok = false;
      const double ljj = sqrt(dj > 0.0 ? dj : 1.0);
      for (int r = j + 1 + lane; r < k; r += 32) {
        double s = L[r * LD + j];
        for (int p = 0; p < j; ++p) s = fma(-L[r * LD + p], L[j * LD + p], s);
        L[r * LD + j] = s / ljj;
      }
      __syncwarp();
      if (lane == 0) L[j * LD + j] = ljj;
      __syncwarp();
    }
    // L y = a (forward), then L^T u = y (backward); one lane per step's
    // updates of the remaining entries
    for (int j = 0; j < k; ++j) {
      if (lane == 0) y[j] = y[j] / L[j * LD + j];
      __syncwarp();
      const double yj = y[j];
      for (int r = j + 1 + lane; r < k; r += 32) y[r] = fma(-L[r * LD + j], yj, y[r]);
      __syncwarp();
    }
    for (int j = k - 1; j >= 0; --j) {
      if (lane == 0) y[j] = y[j] / L[j * LD + j];
      __syncwarp();
      const double yj = y[j];
      for (int r = lane; r < j; r += 32) y[r] = fma(-L[j * LD + r], yj, y[r]);
      __syncwarp();
    }
    for (int l = lane; l < k; l += 32) F[i * k + l] = (TF)y[l];
    if (!ok && lane == 0) atomicOr(err, ERR_NOTCONV);
    __syncwarp();
  }
}

// ------------------------------------------------ f^ over the known entries
// One warp per row; per stored entry the dot u_i . v_j by a warp sum, then
// (x - dot)^2 added by lane 0 in FP64, in entry order.
template <typename TV, typename TF, int KP>
__global__ void __launch_bounds__(NM_T)
nmc_objective_partial(const int64_t* __restrict__ rp, const int32_t* __restrict__ ix,
                      const TV* __restrict__ val, int64_t rows, const TF* __restrict__ U,
                      const TF* __restrict__ V, int k, double scale, double* __restrict__ part) {
  constexpr int E = (KP + 31) / 32;
  __shared__ double sh[NM_T];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t w0 = (int64_t)blockIdx.x * (NM_T / 32) + warp;
  const int64_t nw = (int64_t)gridDim.x * (NM_T / 32);
  double acc = 0.0;
  for (int64_t i = w0; i < rows; i += nw) {
    TF u[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int l = lane + 32 * e;
      u[e] = l < k ? U[i * k + l] : TF(0);
    }
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      const int64_t j = ix[p];
      double d = 0.0;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int l = lane + 32 * e;
        if (l < k) d = fma((double)u[e], (double)V[j * k + l], d);
      }
      d = warp_sum(d);   // every lane holds the dot; lane 0 adds the entry
      const double r = (double)val[p] - d;
      if (lane == 0) acc = fma(r, r * scale, acc);   // scale is a power of two: exact
    }
  }
  const double bs = lanes::block_sum256(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = bs;
}

template <typename TF, int KP>
int pbcd_capacity(int num_sms) {
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, nmc_pbcd_kernel<TF, KP>, NM_T, 0);
  return (per < 1 ? 1 : per) * num_sms;
}

}  // namespace

int nmc_rank_pad(int k) { return k <= 16 ? 16 : k <= 32 ? 32 : k <= 48 ? 48 : 64; }

#define NMC_KP_DISPATCH(kp, F)      \
  do {                              \
    if ((kp) == 16) { F(16); }      \
    else if ((kp) == 32) { F(32); } \
    else if ((kp) == 48) { F(48); } \
    else { F(64); }                 \
  } while (0)

void launch_nmc_gram(const int64_t* rp, const int32_t* ix, const void* val, int64_t rows,
                     const void* B, int k, int fdt, int gdt, void* G, void* A, int num_sms,
                     cudaStream_t s) {
  note_launch(1);
  const int kp = nmc_rank_pad(k);
  int64_t grid = rows < (int64_t)num_sms * 8 ? rows : (int64_t)num_sms * 8;
  if (grid < 1) grid = 1;
#define GL(KPV)                                                                                  \
  if (fdt == T_F64)                                                                              \
    nmc_gram_kernel<double, double, double, KPV><<<(int)grid, NM_T, 0, s>>>(                     \
        rp, ix, (const double*)val, rows, (const double*)B, k, (double*)G, (double*)A);          \
  else if (gdt == T_F64)                                                                         \
    nmc_gram_kernel<float, float, double, KPV><<<(int)grid, NM_T, 0, s>>>(                       \
        rp, ix, (const float*)val, rows, (const float*)B, k, (double*)G, (double*)A);            \
  else                                                                                           \
    nmc_gram_kernel<float, float, float, KPV><<<(int)grid, NM_T, 0, s>>>(                        \
        rp, ix, (const float*)val, rows, (const float*)B, k, (float*)G, (float*)A)
  NMC_KP_DISPATCH(kp, GL);
#undef GL
}

int nmc_pbcd_grid(int fdt, int k, int num_sms, int64_t rows) {
  const int kp = nmc_rank_pad(k);
  int cap = 0;
#define PC(KPV) cap = fdt == T_F64 ? pbcd_capacity<double, KPV>(num_sms) : pbcd_capacity<float, KPV>(num_sms)
  NMC_KP_DISPATCH(kp, PC);
#undef PC
  if (cap > NPART) cap = NPART;
  const int64_t need = (rows + NM_T / 32 - 1) / (NM_T / 32);
  return need < 1 ? 1 : (need < cap ? (int)need : cap);
}

void launch_nmc_pbcd(const NmcArgs& a, int grid, cudaStream_t s) {
  note_launch(1);
  const int kp = nmc_rank_pad(a.k);
  void* args[] = {(void*)&a};
#define PL(KPV)                                                                                 \
  cudaLaunchCooperativeKernel(a.fdt == T_F64 ? (void*)nmc_pbcd_kernel<double, KPV>             \
                                             : (void*)nmc_pbcd_kernel<float, KPV>,              \
                              dim3(grid), dim3(NM_T), args, 0, s)
  NMC_KP_DISPATCH(kp, PL);
#undef PL
}

void launch_nmc_solve(const void* G, const void* A, int64_t rows, int k, double lam, void* F,
                      int fdt, int* err, int num_sms, cudaStream_t s) {
  note_launch(1);
  const int kp = nmc_rank_pad(k);
  int64_t grid = (rows + SV_T / 32 - 1) / (SV_T / 32);
  if (grid > (int64_t)num_sms * 4) grid = (int64_t)num_sms * 4;
  if (grid < 1) grid = 1;
#define SL(KPV)                                                                                 \
  {                                                                                             \
    const size_t smem = sizeof(double) * (SV_T / 32) * ((size_t)KPV * (KPV + 1) + KPV);         \
    if (fdt == T_F64) {                                                                         \
      cudaFuncSetAttribute(nmc_solve_kernel<double, KPV>,                                       \
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);             \
      nmc_solve_kernel<double, KPV><<<(int)grid, SV_T, smem, s>>>(                              \
          (const double*)G, (const double*)A, rows, k, lam, (double*)F, err);                   \
    } else {                                                                                    \
      cudaFuncSetAttribute(nmc_solve_kernel<float, KPV>,                                        \
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);             \
      nmc_solve_kernel<float, KPV><<<(int)grid, SV_T, smem, s>>>(                               \
          (const double*)G, (const double*)A, rows, k, lam, (float*)F, err);                    \
    }                                                                                           \
  }
  NMC_KP_DISPATCH(kp, SL);
#undef SL
}

void launch_nmc_objective(const CsrX& x, const void* U, const void* V, int k, int fdt,
                          double scale, double* part, double* out, cudaStream_t s) {
  note_launch(2);
  const int kp = nmc_rank_pad(k);
#define OL(KPV)                                                                                  \
  if (fdt == T_F64)                                                                              \
    nmc_objective_partial<double, double, KPV><<<NPART, NM_T, 0, s>>>(                           \
        x.row_ptr, x.col, (const double*)x.val, x.m, (const double*)U, (const double*)V, k, scale, part); \
  else                                                                                           \
    nmc_objective_partial<float, float, KPV><<<NPART, NM_T, 0, s>>>(                             \
        x.row_ptr, x.col, (const float*)x.val, x.m, (const float*)U, (const float*)V, k, scale, part)
  NMC_KP_DISPATCH(kp, OL);
#undef OL
  launch_part_reduce(part, 1, out, s);
}

}  // namespace enmf
