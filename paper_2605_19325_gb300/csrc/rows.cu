// Row-local kernels of the eNMF path (the half steps of the iteration are in
// hstep.cu).
//
// Rows are independent here (Sec. 4.2), so each kernel runs one thread per
// factor row, with any r x r matrix it needs staged in shared memory:
//   * stage start of the ascent (Eq. 8/9 step sizes from max(-F));
//   * admm_pass_kernel -- one ADMM pass of Algorithm 1 over W = [U; V];
//   * transforms, negative mass, column sums and the KKT measures (App. G).
// Cost per row is O(r^2); all of these are small next to the O(m n r) sweeps.
#include "internal.h"

namespace enmf {

// ----------------------------------------------------------- stage start
__global__ void state_reset_kernel(DevState* st) {
  st->maxneg_u = 0.0;
  st->maxneg_v = 0.0;
  st->k = 0;
  st->asc_iters = 0;
  st->hals_iters = 0;
  st->negU = 0;
  st->negV = 0;
}

template <typename TF>
__global__ void maxneg_kernel(const TF* __restrict__ F, int64_t total, double* out) {
  __shared__ double sh[256];
  double mx = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    mx = fmax(mx, -(double)F[e]);
  mx = block_max(mx, sh);
  if (threadIdx.x == 0 && mx > 0.0) atomic_max_nonneg(out, mx);
}

__global__ void state_start_kernel(DevState* st, int n_shift) {
  // Eq. 8 / 9 step (reading: max(-F) / (n_shift - 1/2)), fixed for the stage
  st->s_u = st->maxneg_u / ((double)n_shift - 0.5);
  st->s_v = st->maxneg_v / ((double)n_shift - 0.5);
  st->stage = (st->maxneg_u > 0.0 || st->maxneg_v > 0.0) ? 0 : 1;
}

void launch_state_init(const void* U, const void* V, int64_t m, int64_t n, int k, int fdt,
                       int n_shift, DevState* st, double* part, cudaStream_t s) {
  (void)part;
  note_launch(4);
  state_reset_kernel<<<1, 1, 0, s>>>(st);
  int bu = (int)min((int64_t)1024, (m * k + 255) / 256);
  int bv = (int)min((int64_t)1024, (n * k + 255) / 256);
  if (fdt == T_F64) {
    maxneg_kernel<double><<<bu, 256, 0, s>>>((const double*)U, m * k, &st->maxneg_u);
    maxneg_kernel<double><<<bv, 256, 0, s>>>((const double*)V, n * k, &st->maxneg_v);
  } else {
    maxneg_kernel<float><<<bu, 256, 0, s>>>((const float*)U, m * k, &st->maxneg_u);
    maxneg_kernel<float><<<bv, 256, 0, s>>>((const float*)V, n * k, &st->maxneg_v);
  }
  state_start_kernel<<<1, 1, 0, s>>>(st, n_shift);
}

// -------------------------------------------------------------- ADMM pass
constexpr int AP_T = 128;       // threads = rows per tile
constexpr int AP_S = AP_T + 1;  // padded stride of the staged tiles
constexpr int AP_PER_T = (RMAX * RMAX + AP_T - 1) / AP_T;

template <typename TF>
__global__ void __launch_bounds__(AP_T)
admm_pass_kernel(const TF* __restrict__ U, const TF* __restrict__ V, int64_t m, int64_t n, int k,
                 const double* __restrict__ R, TF* __restrict__ Z, TF* __restrict__ Y, double rho_d,
                 int first, DevState* st, double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smraw[];
  TF* Rs = reinterpret_cast<TF*>(smraw);        // k x k
  TF* Ws = Rs + k * k;                          // Ws[j * AP_S + t]
  TF* Bs = Ws + k * AP_S;                       // Bs[j * AP_S + t]
  __shared__ double sh[AP_T];
  if (*(volatile int*)&st->admm_done) return;
  for (int e = threadIdx.x; e < k * k; e += AP_T) Rs[e] = (TF)R[e];
  const TF rho = (TF)rho_d;
  const TF thr = TF(-1) / rho;
  const int64_t rows = m + n;
  const int t = threadIdx.x;
  // W^T B is summed in TF within the block (the pass runs in the form's
  // precision) and in FP64 across blocks.
  TF acc[AP_PER_T];
#pragma unroll
  for (int q = 0; q < AP_PER_T; ++q) acc[q] = TF(0);
  double negm = 0.0;
  for (int64_t t0 = (int64_t)blockIdx.x * AP_T; t0 < rows; t0 += (int64_t)gridDim.x * AP_T) {
    __syncthreads();
    const int64_t i = t0 + t;
    if (i < rows) {
      const TF* w = i < m ? U + i * k : V + (i - m) * k;
      for (int j = 0; j < k; ++j) Ws[j * AP_S + t] = w[j];
      for (int j = 0; j < k; ++j) {
        TF p = TF(0);
        for (int l = 0; l < k; ++l) p = fma(Ws[l * AP_S + t], Rs[l * k + j], p);
        negm += p < TF(0) ? -(double)p : 0.0;
        TF y = Y[i * k + j];
        if (!first) y = y + rho * (Z[i * k + j] - p);   // Y update of Algorithm 1
        TF b = p - y / rho;                             // b = W R - Y / rho
        TF z = b > TF(0) ? b : (b >= thr ? TF(0) : b + TF(1) / rho);   // Eq. 7
        Z[i * k + j] = z;
        Y[i * k + j] = y;
        Bs[j * AP_S + t] = z + y / rho;                 // B = Z + Y / rho
      }
    } else {
      for (int j = 0; j < k; ++j) {
        Ws[j * AP_S + t] = TF(0);
        Bs[j * AP_S + t] = TF(0);
      }
    }
    __syncthreads();
    // M += W_tile^T B_tile
#pragma unroll
    for (int q = 0; q < AP_PER_T; ++q) {
      int e = t + q * AP_T;
      if (e < k * k) {
        int a = e / k, b = e % k;
        TF sacc = acc[q];
        for (int rr = 0; rr < AP_T; ++rr) sacc = fma(Ws[a * AP_S + rr], Bs[b * AP_S + rr], sacc);
        acc[q] = sacc;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < AP_PER_T; ++q) {
    int e = t + q * AP_T;
    if (e < k * k) part[(int64_t)blockIdx.x * k * k + e] = (double)acc[q];
  }
  negm = block_sum(negm, sh);
  if (t == 0) part[(int64_t)NPART * k * k + blockIdx.x] = negm;
}

void launch_admm_pass(const void* U, const void* V, int64_t m, int64_t n, int k, int fdt,
                      const double* R, void* Z, void* Y, double rho, int first, DevState* st,
                      double* part, cudaStream_t s) {
  note_launch(1);
  size_t smem = type_size(fdt) * ((size_t)k * k + 2 * (size_t)k * AP_S);
  if (fdt == T_F64) {
    cudaFuncSetAttribute(admm_pass_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    admm_pass_kernel<double><<<NPART, AP_T, smem, s>>>((const double*)U, (const double*)V, m, n, k, R,
                                                       (double*)Z, (double*)Y, rho, first, st, part);
  } else {
    cudaFuncSetAttribute(admm_pass_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    admm_pass_kernel<float><<<NPART, AP_T, smem, s>>>((const float*)U, (const float*)V, m, n, k, R,
                                                      (float*)Z, (float*)Y, rho, first, st, part);
  }
}

// -------------------------------------------------------- row transforms
constexpr int RT_T = 64;

template <typename TF>
__global__ void __launch_bounds__(RT_T)
row_transform_kernel(const TF* in, int ld_in, int k_in, TF* out, int ld_out, int k_out,
                     int64_t rows, const double* __restrict__ T) {
  extern __shared__ __align__(16) unsigned char smraw[];
  TF* Ts = reinterpret_cast<TF*>(smraw);       // k_in x k_out
  TF* xs = Ts + k_in * k_out;                  // xs[l * RT_T + t]
  for (int e = threadIdx.x; e < k_in * k_out; e += RT_T) Ts[e] = (TF)T[e];
  __syncthreads();
  const int t = threadIdx.x;
  for (int64_t i = (int64_t)blockIdx.x * RT_T + t; i < rows; i += (int64_t)gridDim.x * RT_T) {
    for (int l = 0; l < k_in; ++l) xs[l * RT_T + t] = in[i * ld_in + l];
    for (int j = 0; j < k_out; ++j) {
      TF s = TF(0);
      for (int l = 0; l < k_in; ++l) s = fma(xs[l * RT_T + t], Ts[l * k_out + j], s);
      out[i * ld_out + j] = s;
    }
  }
}

void launch_row_transform(const void* in, int ld_in, int k_in, void* out, int ld_out, int k_out,
                          int64_t rows, int fdt, const double* T, cudaStream_t s) {
  note_launch(1);
  size_t smem = type_size(fdt) * ((size_t)k_in * k_out + (size_t)k_in * RT_T);
  int blocks = (int)min((int64_t)1024, (rows + RT_T - 1) / RT_T);
  if (blocks < 1) blocks = 1;
  if (fdt == T_F64) {
    cudaFuncSetAttribute(row_transform_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    row_transform_kernel<double><<<blocks, RT_T, smem, s>>>((const double*)in, ld_in, k_in, (double*)out,
                                                            ld_out, k_out, rows, T);
  } else {
    cudaFuncSetAttribute(row_transform_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    row_transform_kernel<float><<<blocks, RT_T, smem, s>>>((const float*)in, ld_in, k_in, (float*)out,
                                                           ld_out, k_out, rows, T);
  }
}

// Rows of Y through the orthonormalising map of eig_orth (k x k, see
// small.cu): mode 1 (Tx[2 LMAX]) solves z L^T = y D row by row by forward
// substitution (z_i = (y_i d_i - sum_{p<i} L_ip z_p) / L_ii, in TF, 1 / L_ii
// from Tx), mode 0 multiplies by T.  The row is staged per thread as in
// row_transform_kernel; in place is safe.
template <typename TF>
__global__ void __launch_bounds__(RT_T)
row_orth_kernel(const TF* in, int ld_in, TF* out, int ld_out, int k, int64_t rows,
                const double* __restrict__ T, const double* __restrict__ Tx) {
  extern __shared__ __align__(16) unsigned char smraw[];
  TF* Ts = reinterpret_cast<TF*>(smraw);       // k x k
  TF* ds = Ts + k * k;                         // d (mode 1)
  TF* iv = ds + k;                             // 1 / L_ii (mode 1)
  TF* xs = iv + k;                             // xs[l * RT_T + t]
  const bool tri = Tx[2 * LMAX] != 0.0;
  for (int e = threadIdx.x; e < k * k; e += RT_T) Ts[e] = (TF)T[e];
  for (int e = threadIdx.x; e < k; e += RT_T) {
    ds[e] = (TF)Tx[e];
    iv[e] = (TF)Tx[LMAX + e];
  }
  __syncthreads();
  const int t = threadIdx.x;
  for (int64_t i = (int64_t)blockIdx.x * RT_T + t; i < rows; i += (int64_t)gridDim.x * RT_T) {
    if (tri) {
      for (int l = 0; l < k; ++l) {
        TF sacc = in[i * ld_in + l] * ds[l];
        for (int q = 0; q < l; ++q) sacc = fma(-Ts[l * k + q], xs[q * RT_T + t], sacc);
        xs[l * RT_T + t] = sacc * iv[l];
      }
      for (int j = 0; j < k; ++j) out[i * ld_out + j] = xs[j * RT_T + t];
    } else {
      for (int l = 0; l < k; ++l) xs[l * RT_T + t] = in[i * ld_in + l];
      for (int j = 0; j < k; ++j) {
        TF sacc = TF(0);
        for (int l = 0; l < k; ++l) sacc = fma(xs[l * RT_T + t], Ts[l * k + j], sacc);
        out[i * ld_out + j] = sacc;
      }
    }
  }
}

void launch_row_orth(const void* in, int ld_in, void* out, int ld_out, int k, int64_t rows, int fdt,
                     const double* T, const double* Tx, cudaStream_t s) {
  note_launch(1);
  const size_t smem = type_size(fdt) * ((size_t)k * k + 2 * (size_t)k + (size_t)k * RT_T);
  int blocks = (int)min((int64_t)1024, (rows + RT_T - 1) / RT_T);
  if (blocks < 1) blocks = 1;
  if (fdt == T_F64) {
    cudaFuncSetAttribute(row_orth_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    row_orth_kernel<double><<<blocks, RT_T, smem, s>>>((const double*)in, ld_in, (double*)out, ld_out, k,
                                                       rows, T, Tx);
  } else {
    cudaFuncSetAttribute(row_orth_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    row_orth_kernel<float><<<blocks, RT_T, smem, s>>>((const float*)in, ld_in, (float*)out, ld_out, k, rows,
                                                      T, Tx);
  }
}

void launch_apply_square(void* F, int64_t rows, int k, int fdt, const double* R, cudaStream_t s) {
  // each thread stages its row before writing, so in place is safe
  launch_row_transform(F, k, k, F, k, k, rows, fdt, R, s);
}

// ------------------------------------------------------------------ casts
template <typename TI, typename TO>
__global__ void cast_kernel(const TI* __restrict__ in, TO* __restrict__ out, int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (TO)in[e];
}

void launch_cast(const void* in, int in_dt, void* out, int out_dt, int64_t count, cudaStream_t s) {
  note_launch(1);
  int blocks = (int)min((int64_t)2048, (count + 255) / 256);
  if (blocks < 1) blocks = 1;
  if (in_dt == T_F32 && out_dt == T_F64)
    cast_kernel<float, double><<<blocks, 256, 0, s>>>((const float*)in, (double*)out, count);
  else if (in_dt == T_F64 && out_dt == T_F32)
    cast_kernel<double, float><<<blocks, 256, 0, s>>>((const double*)in, (float*)out, count);
}

// ----------------------------------------------------- small reductions
template <typename TF>
__global__ void __launch_bounds__(256)
negmass_partial(const TF* __restrict__ F, int64_t total, double* part) {
  __shared__ double sh[256];
  const int64_t chunk = (total + NPART - 1) / NPART;
  const int64_t e0 = (int64_t)blockIdx.x * chunk, e1 = min(total, e0 + chunk);
  double s = 0.0;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += 256) {
    double v = (double)F[e];
    s += v < 0.0 ? -v : 0.0;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// One warp: lane l sums partials l, l + 32, ... in order, then a fixed xor
// tree (every lane ends with the same sum).
__global__ void part_sum_to(const double* part, int count, double* out, int accumulate) {
  const int lane = threadIdx.x & 31;
  if (threadIdx.x >= 32 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int b = lane; b < count; b += 32) s += __ldcg(part + b);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[0] = accumulate ? out[0] + s : s;
}

void launch_negmass(const void* F, int64_t rows, int k, int fdt, double* part, double* out,
                    int accumulate, cudaStream_t s) {
  note_launch(2);
  if (fdt == T_F64) negmass_partial<double><<<NPART, 256, 0, s>>>((const double*)F, rows * k, part);
  else negmass_partial<float><<<NPART, 256, 0, s>>>((const float*)F, rows * k, part);
  part_sum_to<<<1, 32, 0, s>>>(part, NPART, out, accumulate);
}

template <typename TF>
__global__ void colsum_partial(const TF* __restrict__ F, int64_t rows, int ld, int k, double* part) {
  const int64_t chunk = (rows + NPART - 1) / NPART;
  const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(rows, r0 + chunk);
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double s = 0.0;
    for (int64_t i = r0; i < r1; ++i) s += (double)F[i * ld + j];
    part[(int64_t)blockIdx.x * k + j] = s;
  }
}

__global__ void colsum_reduce(const double* part, int k, double* out) {
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < NPART; ++b) s += part[(int64_t)b * k + j];
    out[j] = s;
  }
}

void launch_colsum(const void* F, int64_t rows, int ld, int k, int fdt, double* part, double* out,
                   cudaStream_t s) {
  note_launch(2);
  if (fdt == T_F64) colsum_partial<double><<<NPART, 128, 0, s>>>((const double*)F, rows, ld, k, part);
  else colsum_partial<float><<<NPART, 128, 0, s>>>((const float*)F, rows, ld, k, part);
  colsum_reduce<<<1, 128, 0, s>>>(part, k, out);
}

// sum over rows of || Y_i Wr - Q_i UrS ||^2 (r columns): one warp per row,
// the row's entries in registers (lane l holds l, l + 32, l + 64), Wr and UrS
// transposed in shared memory in the factor type, one column of the row's
// difference per butterfly sum; squares summed in FP64 in row order per warp.
constexpr int RR_T = 256;
constexpr int RR_E = (LMAX + 31) / 32;

template <typename TF>
__global__ void __launch_bounds__(RR_T)
rr_residual_kernel(const TF* Y, int ldy, int ky, const TF* Q, int ldq, int kq, int64_t rows, int r,
                   const double* __restrict__ Wr, const double* __restrict__ UrS, double* part) {
  extern __shared__ __align__(16) unsigned char smraw[];
  TF* Wt = reinterpret_cast<TF*>(smraw);   // r x ky: Wt[j * ky + l] = Wr(l, j)
  TF* Ut = Wt + r * ky;                    // r x kq
  __shared__ double sh[RR_T];
  for (int e = threadIdx.x; e < ky * r; e += RR_T) Wt[(e % r) * ky + e / r] = (TF)Wr[e];
  for (int e = threadIdx.x; e < kq * r; e += RR_T) Ut[(e % r) * kq + e / r] = (TF)UrS[e];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t chunk = (rows + NPART - 1) / NPART;
  const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(rows, r0 + chunk);
  double acc = 0.0;
  for (int64_t i = r0 + warp; i < r1; i += RR_T / 32) {
    TF y[RR_E], q[RR_E];
#pragma unroll
    for (int e = 0; e < RR_E; ++e) {
      const int l = lane + 32 * e;
      y[e] = l < ky ? Y[i * ldy + l] : TF(0);
      q[e] = l < kq ? Q[i * ldq + l] : TF(0);
    }
    for (int j = 0; j < r; ++j) {
      TF d = TF(0);
#pragma unroll
      for (int e = 0; e < RR_E; ++e) {
        const int l = lane + 32 * e;
        if (l < ky) d = fma(y[e], Wt[j * ky + l], d);
        if (l < kq) d = fma(-q[e], Ut[j * kq + l], d);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
      acc = fma((double)d, (double)d, acc);   // the same in every lane
    }
  }
  if (lane != 0) acc = 0.0;
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

void launch_rr_residual(const void* Y, int ldy, int ky, const void* Q, int ldq, int kq,
                        int64_t rows, int r, int fdt, const double* Wr, const double* UrS,
                        double* part, double* out, cudaStream_t s) {
  note_launch(2);
  if (fdt == T_F64) {
    const size_t smem = sizeof(double) * ((size_t)ky * r + (size_t)kq * r);
    cudaFuncSetAttribute(rr_residual_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    rr_residual_kernel<double><<<NPART, RR_T, smem, s>>>((const double*)Y, ldy, ky, (const double*)Q, ldq, kq, rows, r, Wr, UrS, part);
  } else {
    const size_t smem = sizeof(float) * ((size_t)ky * r + (size_t)kq * r);
    cudaFuncSetAttribute(rr_residual_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    rr_residual_kernel<float><<<NPART, RR_T, smem, s>>>((const float*)Y, ldy, ky, (const float*)Q, ldq, kq, rows, r, Wr, UrS, part);
  }
  part_sum_to<<<1, 32, 0, s>>>(part, NPART, out, 0);
}

// ------------------------------------------------------------- KKT rows
// Per block: min F, min grad, max(grad * F), sum(grad * F), ||P(grad)||^2,
// ||A||^2, ||F G||^2 with grad = F G - A (App. G).
template <typename TF>
__global__ void __launch_bounds__(RT_T)
kkt_rows_kernel(const TF* __restrict__ F, const TF* __restrict__ A, const double* __restrict__ G,
                int64_t rows, int k, double* part) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double* Gs = reinterpret_cast<double*>(smraw);
  __shared__ double sh[RT_T];
  for (int e = threadIdx.x; e < k * k; e += RT_T) Gs[e] = G[e];
  __syncthreads();
  const int64_t chunk = (rows + NPART - 1) / NPART;
  const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(rows, r0 + chunk);
  double mnw = INFINITY, mng = INFINITY, mxp = -INFINITY, sp = 0.0, pg = 0.0, aa = 0.0, fg = 0.0;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += RT_T) {
    for (int j = 0; j < k; ++j) {
      double s = 0.0;
      for (int l = 0; l < k; ++l) s = fma((double)F[i * k + l], Gs[l * k + j], s);
      double a = (double)A[i * k + j], w = (double)F[i * k + j];
      double gr = s - a;
      mnw = fmin(mnw, w);
      mng = fmin(mng, gr);
      mxp = fmax(mxp, gr * w);
      sp += gr * w;
      double p = w > 0.0 ? gr : fmin(0.0, gr);
      pg = fma(p, p, pg);
      aa = fma(a, a, aa);
      fg = fma(s, s, fg);
    }
  }
  double* o = part + (int64_t)blockIdx.x * 8;
  double v;
  v = block_min(mnw, sh); if (threadIdx.x == 0) o[0] = v;
  v = block_min(mng, sh); if (threadIdx.x == 0) o[1] = v;
  v = block_max(mxp, sh); if (threadIdx.x == 0) o[2] = v;
  v = block_sum(sp, sh);  if (threadIdx.x == 0) o[3] = v;
  v = block_sum(pg, sh);  if (threadIdx.x == 0) o[4] = v;
  v = block_sum(aa, sh);  if (threadIdx.x == 0) o[5] = v;
  v = block_sum(fg, sh);  if (threadIdx.x == 0) o[6] = v;
}

__global__ void kkt_reduce(const double* part, double* out) {
  if (threadIdx.x != 0) return;
  double o[7] = {INFINITY, INFINITY, -INFINITY, 0, 0, 0, 0};
  for (int b = 0; b < NPART; ++b) {
    const double* p = part + b * 8;
    o[0] = fmin(o[0], p[0]);
    o[1] = fmin(o[1], p[1]);
    o[2] = fmax(o[2], p[2]);
    for (int q = 3; q < 7; ++q) o[q] += p[q];
  }
  for (int q = 0; q < 7; ++q) out[q] = o[q];
}

void launch_kkt_rows(const void* F, const void* A, const double* G, int64_t rows, int k, int fdt,
                     double* part, double* out, cudaStream_t s) {
  note_launch(2);
  size_t smem = sizeof(double) * (size_t)k * k;
  if (fdt == T_F64)
    kkt_rows_kernel<double><<<NPART, RT_T, smem, s>>>((const double*)F, (const double*)A, G, rows, k, part);
  else
    kkt_rows_kernel<float><<<NPART, RT_T, smem, s>>>((const float*)F, (const float*)A, G, rows, k, part);
  kkt_reduce<<<1, 32, 0, s>>>(part, out);
}

__global__ void kkt_final_kernel(const double* pu, const double* pv, double* out) {
  // out: min_w, min_grad, delta, sigma, pg_norm, pg_rel
  out[0] = fmin(pu[0], pv[0]);
  out[1] = fmin(pu[1], pv[1]);
  out[2] = fmax(pu[2], pv[2]);
  out[3] = pu[3] + pv[3];
  double pg = sqrt(pu[4] + pv[4]);
  double scale = sqrt(pu[5]) + sqrt(pu[6]) + sqrt(pv[5]) + sqrt(pv[6]);
  out[4] = pg;
  out[5] = scale > 0.0 ? pg / scale : 0.0;
}

void launch_kkt_final(const double* pu, const double* pv, double* out, cudaStream_t s) {
  note_launch(1);
  kkt_final_kernel<<<1, 1, 0, s>>>(pu, pv, out);
}

// ---------------------------------------- transform residual (App. F)
// part[b] = sum over block b's rows of ||B_i - A_i T||^2, every entry formed
// in FP64 (A, B: rows x k of the factor type; T: k x k FP64 row-major).
template <typename TF>
__global__ void __launch_bounds__(RT_T)
transform_residual_partial(const TF* __restrict__ A, const TF* __restrict__ B, int64_t rows, int k,
                           const double* __restrict__ T, double* part) {
  __shared__ double Ts[RMAX * RMAX];
  __shared__ double sh[RT_T];
  for (int e = threadIdx.x; e < k * k; e += RT_T) Ts[e] = T[e];
  __syncthreads();
  const int64_t chunk = (rows + NPART - 1) / NPART;
  const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(rows, r0 + chunk);
  double acc = 0.0;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += RT_T) {
    double a[RMAX];
    for (int l = 0; l < k; ++l) a[l] = (double)A[i * k + l];
    for (int j = 0; j < k; ++j) {
      double sacc = (double)B[i * k + j];
      for (int l = 0; l < k; ++l) sacc = fma(-a[l], Ts[l * k + j], sacc);
      acc = fma(sacc, sacc, acc);
    }
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

void launch_transform_residual(const void* A, const void* B, int64_t rows, int k, int fdt,
                               const double* T, double* part, double* out, cudaStream_t s) {
  note_launch(2);
  if (fdt == T_F64)
    transform_residual_partial<double><<<NPART, RT_T, 0, s>>>((const double*)A, (const double*)B,
                                                             rows, k, T, part);
  else
    transform_residual_partial<float><<<NPART, RT_T, 0, s>>>((const float*)A, (const float*)B,
                                                            rows, k, T, part);
  part_sum_to<<<1, 32, 0, s>>>(part, NPART, out, 0);
}

}  // namespace enmf
