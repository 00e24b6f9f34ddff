// Small dense FP64 linear algebra on one CTA: the r x r and l x l steps of the
// method, all by one-sided (Hestenes) Jacobi SVD in shared memory.
//   * polar_kernel     -- R update of Algorithm 1: R = C D^T from the SVD of
//                         M = W^T B (orthogonal Procrustes, Sec. 4.1.2);
//   * eig_orth_kernel  -- orthonormalising transform of a Gram matrix (SVD
//                         start's range finder);
//   * rr_svd_kernel    -- SVD of the Rayleigh-Ritz matrix of the SVD start;
//   * svd_finish / rr_prep -- U* = U_r S^(1/2), V* = V_r S^(1/2) transforms
//                         with the sign rule.
// One-sided Jacobi orthogonalises the columns of A by plane rotations: for a
// column pair (p, q) with a = |a_p|^2, b = |a_q|^2, g = a_p . a_q the rotation
// with t = sign(z) / (|z| + sqrt(1 + z^2)), z = (b - a) / (2 g) makes them
// orthogonal.  Pairs are visited in round-robin order, one warp per pair.
#include "internal.h"

namespace enmf {

constexpr int SM_T = 256;
constexpr int SM_WARPS = SM_T / 32;
constexpr int JAC_MAX_SWEEPS = 40;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Column-major A (rows x Np) and V (Np x Np) in shared memory, Np even (a
// padding column is zero).  Returns the number of sweeps (JAC_MAX_SWEEPS+1 if
// it did not converge).
__device__ int jacobi_osvd(double* A, int rows, int Np, double* V) {
  __shared__ int rotated;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const double tol = 1e-15 * (double)(rows > 8 ? rows : 8);
  int sweep = 0;
  for (; sweep < JAC_MAX_SWEEPS; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int rnd = 0; rnd < Np - 1; ++rnd) {
      for (int pi = warp; pi < Np / 2; pi += SM_WARPS) {
        int p = pi == 0 ? 0 : 1 + (pi - 1 + rnd) % (Np - 1);
        int qj = Np - 1 - pi;
        int q = 1 + (qj - 1 + rnd) % (Np - 1);
        if (p > q) { int tmp = p; p = q; q = tmp; }
        double* ap = A + (size_t)p * rows;
        double* aq = A + (size_t)q * rows;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int i = lane; i < rows; i += 32) {
          al = fma(ap[i], ap[i], al);
          be = fma(aq[i], aq[i], be);
          ga = fma(ap[i], aq[i], ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (ga != 0.0 && fabs(ga) > tol * sqrt(al * be)) {
          double z = (be - al) / (2.0 * ga);
          double t = (z >= 0.0 ? 1.0 : -1.0) / (fabs(z) + sqrt(1.0 + z * z));
          double c = 1.0 / sqrt(1.0 + t * t);
          double s = c * t;
          for (int i = lane; i < rows; i += 32) {
            double x = ap[i], y = aq[i];
            ap[i] = c * x - s * y;
            aq[i] = s * x + c * y;
          }
          double* vp = V + (size_t)p * Np;
          double* vq = V + (size_t)q * Np;
          for (int i = lane; i < Np; i += 32) {
            double x = vp[i], y = vq[i];
            vp[i] = c * x - s * y;
            vq[i] = s * x + c * y;
          }
          if (lane == 0) rotated = 1;
        }
      }
      __syncthreads();
    }
    if (!rotated) break;
    __syncthreads();
  }
  return sweep;
}

// Column norms and the descending order (ties by index).
__device__ void sort_desc(const double* A, int rows, int N, double* nrm, int* ord) {
  for (int c = threadIdx.x; c < N; c += SM_T) {
    double s = 0.0;
    for (int i = 0; i < rows; ++i) s = fma(A[(size_t)c * rows + i], A[(size_t)c * rows + i], s);
    nrm[c] = sqrt(s);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < N; c += SM_T) {
    int rank = 0;
    for (int d = 0; d < N; ++d)
      if (nrm[d] > nrm[c] || (nrm[d] == nrm[c] && d < c)) ++rank;
    ord[rank] = c;
  }
  __syncthreads();
}

__device__ void set_identity(double* V, int Np) {
  for (int e = threadIdx.x; e < Np * Np; e += SM_T) V[e] = (e / Np == e % Np) ? 1.0 : 0.0;
}

// ------------------------------------------------------------- polar (R)
// M (k x k row-major) -> R = C D^T with M = C S D^T.  With the one-sided
// Jacobi on the columns of M: M V = A (orthogonal columns), so C = A S^-1 and
// D = V, R = sum_c (a_c / s_c) v_c^T.
__global__ void __launch_bounds__(SM_T)
polar_kernel(const double* __restrict__ Mg, int k, double* R, double tol, DevState* st, int* err) {
  extern __shared__ double smd[];
  __shared__ double red[SM_T];
  if (*(volatile int*)&st->admm_done) return;
  const int Np = k + (k & 1);
  double* A = smd;                 // Np columns x k rows (column-major)
  double* V = A + (size_t)Np * k;  // Np x Np
  double* nrm = V + (size_t)Np * Np;
  double* Rn = nrm + Np;           // k x k
  int* ord = reinterpret_cast<int*>(Rn + (size_t)k * k);
  for (int e = threadIdx.x; e < Np * k; e += SM_T) {
    int c = e / k, i = e % k;
    A[e] = c < k ? Mg[i * k + c] : 0.0;   // column c of M
  }
  set_identity(V, Np);
  __syncthreads();
  int sw = jacobi_osvd(A, k, Np, V);
  sort_desc(A, k, Np, nrm, ord);
  // R_ij = sum_c A_ic V_jc / s_c over c < k (singular values of M)
  double smin = nrm[ord[k - 1]];
  for (int e = threadIdx.x; e < k * k; e += SM_T) {
    int i = e / k, j = e % k;
    double s = 0.0;
    for (int c = 0; c < Np; ++c)
      if (nrm[c] > 0.0) s = fma(A[(size_t)c * k + i] / nrm[c], V[(size_t)c * Np + j], s);
    Rn[e] = s;
  }
  __syncthreads();
  double d = 0.0;
  for (int e = threadIdx.x; e < k * k; e += SM_T) {
    double x = Rn[e] - R[e];
    d = fma(x, x, d);
  }
  d = block_sum(d, red);
  for (int e = threadIdx.x; e < k * k; e += SM_T) R[e] = Rn[e];
  if (threadIdx.x == 0) {
    double dR = sqrt(d);
    st->dR = dR;
    st->admm_steps += 1;
    if (sw > JAC_MAX_SWEEPS - 1 || !(smin > 0.0)) atomicOr(err, ERR_NOTCONV);
    if (dR <= tol * sqrt((double)k)) st->admm_done = 1;
  }
}

static size_t small_smem(int rows, int Np) {
  return sizeof(double) * ((size_t)Np * rows + (size_t)Np * Np + Np + (size_t)Np * Np) +
         sizeof(int) * Np + 64;
}

void launch_polar(const double* M, int k, double* R, double* R_prev, double tol, DevState* st,
                  int* err, cudaStream_t s) {
  (void)R_prev;
  int Np = k + (k & 1);
  size_t smem = small_smem(k, Np);
  cudaFuncSetAttribute(polar_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  polar_kernel<<<1, SM_T, smem, s>>>(M, k, R, tol, st, err);
}

// ------------------------------------------------------ Gram -> orth map
// G (k x k, symmetric PSD).  One-sided Jacobi on its columns gives G V = A
// with orthogonal columns; for PSD G the columns of V are eigenvectors and
// |a_c| the eigenvalues.  T = V_kept diag(lambda^-1/2) for lambda > tau *
// lambda_max (dropped directions give zero columns).
__global__ void __launch_bounds__(SM_T)
eig_orth_kernel(const double* __restrict__ G, int k, double tau, double* T, int* kept, int* err) {
  extern __shared__ double smd[];
  const int Np = k + (k & 1);
  double* A = smd;
  double* V = A + (size_t)Np * k;
  double* nrm = V + (size_t)Np * Np;
  int* ord = reinterpret_cast<int*>(nrm + Np + (size_t)Np * Np);
  for (int e = threadIdx.x; e < Np * k; e += SM_T) {
    int c = e / k, i = e % k;
    A[e] = c < k ? G[i * k + c] : 0.0;
  }
  set_identity(V, Np);
  __syncthreads();
  int sw = jacobi_osvd(A, k, Np, V);
  sort_desc(A, k, Np, nrm, ord);
  const double lmax = nrm[ord[0]];
  for (int e = threadIdx.x; e < k * k; e += SM_T) {
    int i = e / k, j = e % k;
    int c = ord[j];
    double lam = nrm[c];
    T[e] = (lmax > 0.0 && lam > tau * lmax) ? V[(size_t)c * Np + i] / sqrt(lam) : 0.0;
  }
  if (threadIdx.x == 0) {
    int cnt = 0;
    for (int j = 0; j < k; ++j)
      if (lmax > 0.0 && nrm[ord[j]] > tau * lmax) ++cnt;
    *kept = cnt;
    if (sw > JAC_MAX_SWEEPS - 1) atomicOr(err, ERR_NOTCONV);
  }
}

void launch_eig_orth(const double* G, int k, double tau, double* T, int* kept, int* err,
                     cudaStream_t s) {
  int Np = k + (k & 1);
  size_t smem = small_smem(k, Np);
  cudaFuncSetAttribute(eig_orth_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  eig_orth_kernel<<<1, SM_T, smem, s>>>(G, k, tau, T, kept, err);
}

// ------------------------------------------------------ Rayleigh-Ritz SVD
// P = Q2^T Bt (k2 x k1, row-major).  The Rayleigh-Ritz matrix is
// B = Q^T X = P^T Q2^T, and P^T (k1 x k2) = Ut S Wt^T.  Column c of P^T is
// row c of P, so P's memory is P^T in column-major order.
__global__ void __launch_bounds__(SM_T)
rr_svd_kernel(const double* __restrict__ P, int k2, int k1, double* sigma, double* Ut, double* Wt,
              int* err) {
  extern __shared__ double smd[];
  const int Np = k2 + (k2 & 1);
  double* A = smd;                  // Np columns x k1 rows
  double* V = A + (size_t)Np * k1;  // Np x Np
  double* nrm = V + (size_t)Np * Np;
  int* ord = reinterpret_cast<int*>(nrm + Np + (size_t)Np * Np);
  for (int e = threadIdx.x; e < Np * k1; e += SM_T) {
    int c = e / k1, i = e % k1;
    A[e] = c < k2 ? P[(size_t)c * k1 + i] : 0.0;
  }
  set_identity(V, Np);
  __syncthreads();
  int sw = jacobi_osvd(A, k1, Np, V);
  sort_desc(A, k1, Np, nrm, ord);
  for (int j = threadIdx.x; j < k2; j += SM_T) sigma[j] = nrm[ord[j]];
  for (int e = threadIdx.x; e < k1 * k2; e += SM_T) {
    int i = e / k2, j = e % k2;
    int c = ord[j];
    Ut[e] = nrm[c] > 0.0 ? A[(size_t)c * k1 + i] / nrm[c] : 0.0;
  }
  for (int e = threadIdx.x; e < k2 * k2; e += SM_T) {
    int i = e / k2, j = e % k2;
    Wt[e] = V[(size_t)ord[j] * Np + i];
  }
  if (threadIdx.x == 0 && sw > JAC_MAX_SWEEPS - 1) atomicOr(err, ERR_NOTCONV);
}

void launch_rr_svd(const double* P, int k2, int k1, double* sigma, double* Ut, double* Wt,
                   int* err, cudaStream_t s) {
  int Np = k2 + (k2 & 1);
  size_t smem = small_smem(k1 > Np ? k1 : Np, Np);
  cudaFuncSetAttribute(rr_svd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  rr_svd_kernel<<<1, SM_T, smem, s>>>(P, k2, k1, sigma, Ut, Wt, err);
}

// Residual inputs: Wr = Wt[:, :r] (k2 x r), UrS = Ut[:, :r] S_r (k1 x r).
__global__ void rr_prep_kernel(const double* sigma, const double* Ut, const double* Wt, int k1,
                               int k2, int r, double* Wr, double* UrS, DevState* st) {
  for (int e = threadIdx.x; e < k2 * r; e += blockDim.x) Wr[e] = Wt[(e / r) * k2 + e % r];
  for (int e = threadIdx.x; e < k1 * r; e += blockDim.x)
    UrS[e] = Ut[(e / r) * k2 + e % r] * sigma[e % r];
  if (threadIdx.x == 0) st->sigma1 = sigma[0];
}

void launch_rr_prep(const double* sigma, const double* Ut, const double* Wt, int k1, int k2,
                    int r, double* Wr, double* UrS, DevState* st, cudaStream_t s) {
  rr_prep_kernel<<<1, 256, 0, s>>>(sigma, Ut, Wt, k1, k2, r, Wr, UrS, st);
}

// U* = Q Tu, V* = Q2 Tv with Tu = Ut_r S^(1/2), Tv = Wt_r S^(1/2), column j of
// both negated when colsum(U*)_j + colsum(V*)_j < 0 (sign reading of the
// SVD start).
__global__ void svd_finish_kernel(const double* sigma, const double* Ut, const double* Wt, int k1,
                                  int k2, int r, const double* csQ, const double* csQ2, double* Tu,
                                  double* Tv, double* sigma_out) {
  __shared__ double sgn[RMAX];
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    double rt = sqrt(sigma[j]);
    double s = 0.0;
    for (int i = 0; i < k1; ++i) s += csQ[i] * Ut[i * k2 + j] * rt;
    for (int i = 0; i < k2; ++i) s += csQ2[i] * Wt[i * k2 + j] * rt;
    sgn[j] = s < 0.0 ? -1.0 : 1.0;
    if (sigma_out) sigma_out[j] = sigma[j];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < k1 * r; e += blockDim.x) {
    int i = e / r, j = e % r;
    Tu[e] = Ut[i * k2 + j] * sqrt(sigma[j]) * sgn[j];
  }
  for (int e = threadIdx.x; e < k2 * r; e += blockDim.x) {
    int i = e / r, j = e % r;
    Tv[e] = Wt[i * k2 + j] * sqrt(sigma[j]) * sgn[j];
  }
}

void launch_svd_finish(const double* sigma, const double* Ut, const double* Wt, int k1, int k2,
                       int r, const double* colsumQ, const double* colsumQ2, double* Tu,
                       double* Tv, double* sigma_out, cudaStream_t s) {
  svd_finish_kernel<<<1, 256, 0, s>>>(sigma, Ut, Wt, k1, k2, r, colsumQ, colsumQ2, Tu, Tv,
                                      sigma_out);
}

}  // namespace enmf
