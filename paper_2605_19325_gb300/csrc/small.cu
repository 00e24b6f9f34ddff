// Small dense FP64 linear algebra on one CTA: the r x r and l x l steps of the
// method, in shared memory, mostly by one-sided (Hestenes) Jacobi SVD.
//   * polar_kernel     -- R update of Algorithm 1 with FP64 factors: R = C D^T
//                         from the SVD of M = W^T B (orthogonal Procrustes,
//                         Sec. 4.1.2); the FP32 forms use admm.cu;
//   * eig_orth_kernel  -- orthonormalising transform of a Gram matrix (SVD
//                         start's range finder): scaled Cholesky, or the
//                         Jacobi eigen map when the Gram is near singular;
//   * rr_svd_kernel    -- SVD of the Rayleigh-Ritz matrix of the SVD start;
//   * svd_finish / rr_prep -- U* = U_r S^(1/2), V* = V_r S^(1/2) transforms
//                         with the sign rule.
// One-sided Jacobi orthogonalises the columns of A by plane rotations: for a
// column pair (p, q) with a = |a_p|^2, b = |a_q|^2, g = a_p . a_q the rotation
// with t = sign(z) / (|z| + sqrt(1 + z^2)), z = (b - a) / (2 g) makes them
// orthogonal.  Pairs are visited in round-robin order, one warp per pair.
#include "internal.h"

namespace enmf {

constexpr int SM_T = 1024;   // one warp per column pair of a round (up to 32 pairs)
constexpr int SM_WARPS = SM_T / 32;
constexpr int JAC_MAX_SWEEPS = 40;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Column pair of slot pi in round rnd of the round-robin (circle) ordering:
// every pair of the Np columns meets once per sweep, and the pairs of a round
// are disjoint.
__device__ __forceinline__ void rr_pair(int pi, int rnd, int Np, int& p, int& q) {
  p = pi == 0 ? 0 : 1 + (pi - 1 + rnd) % (Np - 1);
  q = 1 + (Np - 2 - pi + rnd) % (Np - 1);
  if (p > q) { int t = p; p = q; q = t; }
}

// Scratch of the Jacobi rounds, shared by its FP32 and FP64 instances (one
// allocation per kernel).
__shared__ int jac_rotated;
__shared__ double jac_part[LMAX / 2][3][33];
__shared__ double jac_rot[LMAX / 2][2];

// Column-major A (rows x Np) and V (Np x Np) in shared memory, Np even (a
// padding column is zero), rows <= LMAX, Np <= LMAX.  Runs at most
// max_sweeps sweeps and returns the number run.  A pair is rotated when
// |a_p . a_q| > tol * |a_p| |a_q|, tol = (1e-15 in FP64, 1e-6 in FP32) x
// max(rows, 8): above the rounding of the dot products, so the sweeps end.
//
// FP64 issue rate is the limit on this GPU, so each round keeps the FP64
// instruction count low: lanes form partial products of their rows, one
// thread per (pair, quantity) sums the 32 partials in lane order, one thread
// per pair computes the rotation, then one warp per pair applies it.
template <typename T>
__device__ int jacobi_osvd(T* A, int rows, int Np, T* V, int max_sweeps) {
  T (*part)[3][33] = reinterpret_cast<T (*)[3][33]>(jac_part);
  T (*rot)[2] = reinterpret_cast<T (*)[2]>(jac_rot);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int npairs = Np / 2;
  const T tol = (T)((sizeof(T) == 8 ? 1e-15 : 1e-6) * (double)(rows > 8 ? rows : 8));
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) jac_rotated = 0;
    for (int rnd = 0; rnd < Np - 1; ++rnd) {
      // partial products: lane l takes rows l, l + 32, ...
      for (int pi = warp; pi < npairs; pi += SM_WARPS) {
        int p, q;
        rr_pair(pi, rnd, Np, p, q);
        const T* ap = A + (size_t)p * rows;
        const T* aq = A + (size_t)q * rows;
        T al = 0, be = 0, ga = 0;
        for (int i = lane; i < rows; i += 32) {
          const T x = ap[i], y = aq[i];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
        part[pi][0][lane] = al;
        part[pi][1][lane] = be;
        part[pi][2][lane] = ga;
      }
      __syncthreads();
      // one thread per (pair, quantity): fixed lane-order sum
      for (int t = threadIdx.x; t < 3 * npairs; t += SM_T) {
        const int pi = t / 3, qq = t % 3;
        T s = 0;
#pragma unroll 8
        for (int l = 0; l < 32; ++l) s += part[pi][qq][l];
        part[pi][qq][32] = s;
      }
      __syncthreads();
      // one thread per pair: the rotation (c, s), or (1, 0) when the pair is
      // already orthogonal to working precision
      for (int pi = threadIdx.x; pi < npairs; pi += SM_T) {
        const T al = part[pi][0][32], be = part[pi][1][32], ga = part[pi][2][32];
        T c = 1, s = 0;
        if (ga != T(0) && fabs(ga) > tol * sqrt(al * be)) {
          const T z = (be - al) / (T(2) * ga);
          const T t = (z >= T(0) ? T(1) : T(-1)) / (fabs(z) + sqrt(T(1) + z * z));
          c = T(1) / sqrt(T(1) + t * t);
          s = c * t;
          jac_rotated = 1;
        }
        rot[pi][0] = c;
        rot[pi][1] = s;
      }
      __syncthreads();
      for (int pi = warp; pi < npairs; pi += SM_WARPS) {
        const T c = rot[pi][0], s = rot[pi][1];
        if (s == T(0)) continue;
        int p, q;
        rr_pair(pi, rnd, Np, p, q);
        T* ap = A + (size_t)p * rows;
        T* aq = A + (size_t)q * rows;
        for (int i = lane; i < rows; i += 32) {
          const T x = ap[i], y = aq[i];
          ap[i] = c * x - s * y;
          aq[i] = s * x + c * y;
        }
        T* vp = V + (size_t)p * Np;
        T* vq = V + (size_t)q * Np;
        for (int i = lane; i < Np; i += 32) {
          const T x = vp[i], y = vq[i];
          vp[i] = c * x - s * y;
          vq[i] = s * x + c * y;
        }
      }
      __syncthreads();
    }
    if (!jac_rotated) break;
    __syncthreads();
  }
  return sweep;
}

// FP32 instance, where the FP32 rate leaves the syncs as the cost: one warp
// per pair of a round forms the three dot products (a fixed xor tree, so
// every lane holds the same sums), computes the rotation and applies it, and
// a round is one __syncthreads.  The same rotation rule and tolerance as
// jacobi_osvd.
__device__ int jacobi_osvd_f32(float* A, int rows, int Np, float* V, int max_sweeps) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int npairs = Np / 2;
  const float tol = 1e-6f * (float)(rows > 8 ? rows : 8);
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) jac_rotated = 0;
    __syncthreads();
    for (int rnd = 0; rnd < Np - 1; ++rnd) {
      for (int pi = warp; pi < npairs; pi += SM_WARPS) {
        int p, q;
        rr_pair(pi, rnd, Np, p, q);
        float* ap = A + (size_t)p * rows;
        float* aq = A + (size_t)q * rows;
        float al = 0.f, be = 0.f, ga = 0.f;
        for (int i = lane; i < rows; i += 32) {
          const float x = ap[i], y = aq[i];
          al = fmaf(x, x, al);
          be = fmaf(y, y, be);
          ga = fmaf(x, y, ga);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        if (ga != 0.f && fabsf(ga) > tol * sqrtf(al * be)) {
          const float z = (be - al) / (2.f * ga);
          const float t = (z >= 0.f ? 1.f : -1.f) / (fabsf(z) + sqrtf(1.f + z * z));
          const float c = 1.f / sqrtf(1.f + t * t);
          const float sn = c * t;
          if (lane == 0) jac_rotated = 1;
          for (int i = lane; i < rows; i += 32) {
            const float x = ap[i], y = aq[i];
            ap[i] = c * x - sn * y;
            aq[i] = sn * x + c * y;
          }
          float* vp = V + (size_t)p * Np;
          float* vq = V + (size_t)q * Np;
          for (int i = lane; i < Np; i += 32) {
            const float x = vp[i], y = vq[i];
            vp[i] = c * x - sn * y;
            vq[i] = sn * x + c * y;
          }
        }
      }
      __syncthreads();
    }
    if (!jac_rotated) break;
    __syncthreads();
  }
  return sweep;
}

// The same one-sided Jacobi in two precisions: sweeps in FP32 (64 times the
// FP64 rate on this GPU) to single-precision orthogonality of A's columns,
// then the accumulated rotation V32 -- orthogonal only to FP32 rounding -- is
// made orthogonal in FP64 by one Newton-Schulz step V = V32 (3 I - V32^T V32)
// / 2, A = A0 V is formed in FP64, and FP64 sweeps finish: from nearly
// orthogonal columns they converge in one or two sweeps (Jacobi's quadratic
// convergence).  A (FP64, in/out) as in jacobi_osvd, V (FP64, out) the
// accumulated rotation; scratch: A32 (Np x rows floats), V32 (Np x Np
// floats), T (Np x Np doubles).  Returns the FP64 sweeps run.
__device__ int jacobi_osvd_mixed(double* A, int rows, int Np, double* V, float* A32, float* V32,
                                 double* T) {
  for (int e = threadIdx.x; e < Np * rows; e += SM_T) A32[e] = (float)A[e];
  for (int e = threadIdx.x; e < Np * Np; e += SM_T) V32[e] = (e / Np == e % Np) ? 1.f : 0.f;
  __syncthreads();
  jacobi_osvd_f32(A32, rows, Np, V32, JAC_MAX_SWEEPS);
  // two Newton-Schulz steps V <- V (3 I - V^T V) / 2 in FP64 from V = V32
  // (an orthogonality error e becomes about e^2 per step); V^T V goes to T,
  // the new V to registers first (column-major: V[c * Np + i] is entry (i, c))
  constexpr int NV = (LMAX * LMAX + SM_T - 1) / SM_T;   // entries per thread
  for (int e = threadIdx.x; e < Np * Np; e += SM_T) V[e] = (double)V32[e];
  __syncthreads();
  for (int step = 0; step < 2; ++step) {
    for (int e = threadIdx.x; e < Np * Np; e += SM_T) {   // T = V^T V
      const int c = e / Np, i = e % Np;
      double acc = 0.0;
      for (int j = 0; j < Np; ++j) acc = fma(V[(size_t)i * Np + j], V[(size_t)c * Np + j], acc);
      T[e] = acc;
    }
    __syncthreads();
    double nv[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const int e = threadIdx.x + q * SM_T;
      if (e < Np * Np) {
        const int c = e / Np, i = e % Np;
        double acc = 0.0;
        for (int j = 0; j < Np; ++j) acc = fma(V[(size_t)j * Np + i], T[(size_t)c * Np + j], acc);
        nv[q] = 1.5 * V[e] - 0.5 * acc;
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const int e = threadIdx.x + q * SM_T;
      if (e < Np * Np) V[e] = nv[q];
    }
    __syncthreads();
  }
  // T = A0 V (column c of T = sum_j column j of A0 times V(j, c)), then A = T
  for (int e = threadIdx.x; e < Np * rows; e += SM_T) {
    const int c = e / rows, i = e % rows;
    double acc = 0.0;
    for (int j = 0; j < Np; ++j) acc = fma(A[(size_t)j * rows + i], V[(size_t)c * Np + j], acc);
    T[e] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < Np * rows; e += SM_T) A[e] = T[e];
  __syncthreads();
  return jacobi_osvd<double>(A, rows, Np, V, JAC_MAX_SWEEPS);
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
// Warm start: successive ADMM steps change M little, so the rotation starts
// from the previous step's right singular vectors D (Np x Np column-major,
// identity at the first step): A = M D is already nearly column-orthogonal and
// the sweeps converge in a few passes.  D is updated in place.
// Shared part of the polar kernels: Rn (k x k, shared) = polar(Mg), D (Np x
// Np, global, column-major) the warm start, updated.  Returns the Jacobi
// sweeps run; *smin_out the smallest singular value of M.
__device__ int polar_core(const double* __restrict__ Mg, int k, double* D, double* smd,
                          double*& Rn_out, double* smin_out) {
  const int Np = k + (k & 1);
  double* A = smd;                 // Np columns x k rows (column-major)
  double* V = A + (size_t)Np * k;  // Np x Np
  double* nrm = V + (size_t)Np * Np;
  double* Rn = nrm + Np;           // k x k
  double* Ms = Rn + (size_t)k * k; // k x k
  for (int e = threadIdx.x; e < k * k; e += SM_T) Ms[e] = Mg[e];
  for (int e = threadIdx.x; e < Np * Np; e += SM_T) V[e] = D[e];
  __syncthreads();
  for (int e = threadIdx.x; e < Np * k; e += SM_T) {
    int c = e / k, i = e % k;      // A_ic = sum_j M_ij V_jc (padding row/column of V is e_k)
    double s = 0.0;
    for (int j = 0; j < k; ++j) s = fma(Ms[i * k + j], V[(size_t)c * Np + j], s);
    A[e] = s;
  }
  __syncthreads();
  int sw = jacobi_osvd<double>(A, k, Np, V, JAC_MAX_SWEEPS);
  for (int c = threadIdx.x; c < Np; c += SM_T) {
    double s = 0.0;
    for (int i = 0; i < k; ++i) s = fma(A[(size_t)c * k + i], A[(size_t)c * k + i], s);
    nrm[c] = sqrt(s);
  }
  for (int e = threadIdx.x; e < Np * Np; e += SM_T) D[e] = V[e];
  __syncthreads();
  // R_ij = sum_c A_ic V_jc / s_c over the k singular values of M (the
  // padding column, if any, has s = 0 and is skipped)
  double smin = INFINITY;
  for (int c = 0; c < Np; ++c)
    if (!(k & 1) || c != k) smin = fmin(smin, nrm[c]);
  for (int e = threadIdx.x; e < Np * k; e += SM_T) {   // C = A S^-1, one division per column
    const int c = e / k;
    const double inv = nrm[c] > 0.0 ? 1.0 / nrm[c] : 0.0;
    A[e] *= inv;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < k * k; e += SM_T) {
    int i = e / k, j = e % k;
    double s = 0.0;
    for (int c = 0; c < Np; ++c) s = fma(A[(size_t)c * k + i], V[(size_t)c * Np + j], s);
    Rn[e] = s;
  }
  __syncthreads();
  Rn_out = Rn;
  *smin_out = smin;
  return sw;
}

// ------------------------------------------------------------- polar (R)
// M (k x k row-major) -> R = C D^T with M = C S D^T.  With the one-sided
// Jacobi on the columns of M: M V = A (orthogonal columns), so C = A S^-1 and
// D = V, R = sum_c (a_c / s_c) v_c^T.
// Warm start: successive ADMM steps change M little, so the rotation starts
// from the previous step's right singular vectors D (Np x Np column-major,
// identity at the first step): A = M D is already nearly column-orthogonal and
// the sweeps converge in a few passes.  D is updated in place.
__global__ void __launch_bounds__(SM_T)
polar_kernel(const double* __restrict__ Mg, int k, double* R, double* D, double tol, DevState* st,
             int* err) {
  extern __shared__ double smd[];
  __shared__ double red[SM_T];
  if (*(volatile int*)&st->admm_done) return;
  double* Rn;
  double smin;
  const int sw = polar_core(Mg, k, D, smd, Rn, &smin);
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
    st->jac_sweeps = sw;
    if (sw > JAC_MAX_SWEEPS - 1 || !(smin > 0.0)) atomicOr(err, ERR_NOTCONV);
    if (dR <= tol * sqrt((double)k)) st->admm_done = 1;
  }
}

// The same polar factor into Rout, with no loop bookkeeping (Algorithm 4's
// R1 and R2 updates, each with its own warm start D).  Algorithm 4 runs two
// warm-started factors for hundreds of steps, and the rounding of the
// accumulated Jacobi rotations drifts D (and so R) away from orthogonality
// by about 1e-12 at r = 49; one Newton-Schulz step R (3I - R^T R) / 2 maps an
// R with |R^T R - I| = e to one with about 3e^2 / 4 and leaves the polar
// factor itself unchanged.
__global__ void __launch_bounds__(SM_T)
polar_plain_kernel(const double* __restrict__ Mg, int k, double* Rout, double* D, int* err) {
  extern __shared__ double smd[];
  double* Rn;
  double smin;
  const int sw = polar_core(Mg, k, D, smd, Rn, &smin);
  double* P = Rn + (size_t)k * k;  // the input copy's slot, free again
  for (int e = threadIdx.x; e < k * k; e += SM_T) {   // P = R^T R
    const int i = e / k, j = e % k;
    double s = 0.0;
    for (int c = 0; c < k; ++c) s = fma(Rn[c * k + i], Rn[c * k + j], s);
    P[e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < k * k; e += SM_T) {   // R (3I - P) / 2
    const int i = e / k, j = e % k;
    double s = 0.0;
    for (int c = 0; c < k; ++c) s = fma(Rn[i * k + c], (c == j ? 3.0 : 0.0) - P[c * k + j], s);
    Rout[e] = 0.5 * s;
  }
  if (threadIdx.x == 0 && (sw > JAC_MAX_SWEEPS - 1 || !(smin > 0.0))) atomicOr(err, ERR_NOTCONV);
}

static size_t small_smem(int rows, int Np) {
  return sizeof(double) * ((size_t)Np * rows + (size_t)Np * Np + Np + (size_t)Np * Np) +
         sizeof(int) * Np + 64;
}

void launch_polar(const double* M, int k, double* R, double* D, double tol, DevState* st,
                  int* err, cudaStream_t s) {
  note_launch(1);
  int Np = k + (k & 1);
  size_t smem = sizeof(double) * ((size_t)Np * k + (size_t)Np * Np + Np + 2 * (size_t)k * k) + 64;
  cudaFuncSetAttribute(polar_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  polar_kernel<<<1, SM_T, smem, s>>>(M, k, R, D, tol, st, err);
}

void launch_polar_plain(const double* M, int k, double* R, double* D, int* err, cudaStream_t s) {
  note_launch(1);
  int Np = k + (k & 1);
  size_t smem = sizeof(double) * ((size_t)Np * k + (size_t)Np * Np + Np + 2 * (size_t)k * k) + 64;
  cudaFuncSetAttribute(polar_plain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  polar_plain_kernel<<<1, SM_T, smem, s>>>(M, k, R, D, err);
}

// ------------------------------------------------------ Gram -> orth map
// G = Y^T Y (k x k, symmetric PSD) -> the map with Y T orthonormal, applied
// to the rows of Y by row_orth (rows.cu).
//
// Fast path, scaled Cholesky: with D = diag(G)^-1/2 and D G D = L L^T the map
// is T = D L^-T (then (Y T)^T (Y T) = L^-1 D G D L^-T = I); it is not formed:
// T receives L (row-major, lower triangle and diagonal) and Tx the diagonal of
// D (Tx[0..k)), 1 / L_jj (Tx[LMAX..LMAX+k)) and the mode 1 (Tx[2 LMAX]), and
// each row y of Y is mapped by the triangular solve  z L^T = y D.  It is taken
// when every pivot of D G D is above tau (the diagonal is 1 after scaling),
// i.e. Y has no direction near the truncation threshold; the caller runs two
// passes, so the orthogonality lost to cond(G) in the first is restored by
// the second.
//
// Otherwise (a pivot at or below tau: Y numerically rank deficient), the
// eigen path: one-sided Jacobi on the columns of G gives G V = A with
// orthogonal columns; for PSD G the columns of V are eigenvectors and |a_c|
// the eigenvalues.  T = V_kept diag(lambda^-1/2) for lambda > tau *
// lambda_max (dropped directions give zero columns), mode 0 (a product).
//
// 1 / sqrt(d), d > 0: an FP32 estimate refined by two Newton-Raphson steps
// for the reciprocal square root, y <- y (3 - d y^2) / 2 (each step about
// doubles the correct bits, 24 -> 48 -> FP64).  A dependent FP64 operation
// costs on the order of a hundred cycles on this GPU; this chain is far
// shorter than a square root followed by a division.
__device__ __forceinline__ double rsqrt_nr(double d) {
  if (!(d >= 1e-30 && d <= 1e30)) return 1.0 / sqrt(d);   // outside the FP32 start's range
  double y = (double)rsqrtf((float)d);
  y = y * (1.5 - 0.5 * d * y * y);
  y = y * (1.5 - 0.5 * d * y * y);
  return y;
}

__device__ bool chol_orth(const double* __restrict__ G, int k, double tau, double* C,
                          double* dsc, double* T, double* Tx) {
  __shared__ int ok;
  __shared__ double invd[LMAX];
  if (threadIdx.x == 0) ok = 1;
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += SM_T) {
    const double g = G[i * k + i];
    if (!(g > 0.0)) ok = 0;
    dsc[i] = g > 0.0 ? rsqrt_nr(g) : 0.0;
  }
  __syncthreads();
  if (!ok) return false;
  for (int e = threadIdx.x; e < k * k; e += SM_T) {
    const int i = e / k, j = e % k;
    C[e] = G[e] * dsc[i] * dsc[j];
  }
  __syncthreads();
  // right-looking Cholesky, lower triangle of C (row-major) becomes L; the
  // column is scaled by the reciprocal of its pivot (a multiplication)
  for (int j = 0; j < k; ++j) {
    if (threadIdx.x == 0) {
      const double d = C[j * k + j];
      if (d > tau) {
        const double y = rsqrt_nr(d);
        C[j * k + j] = d * y;
        invd[j] = y;
      } else {
        ok = 0;
      }
    }
    __syncthreads();
    if (!ok) return false;
    const double inv = invd[j];
    for (int i = j + 1 + threadIdx.x; i < k; i += SM_T) C[i * k + j] *= inv;
    __syncthreads();
    const int w = k - j - 1;   // trailing block (j+1 .. k-1), lower triangle
    for (int e = threadIdx.x; e < w * w; e += SM_T) {
      const int i = j + 1 + e / w, c = j + 1 + e % w;
      if (c <= i) C[i * k + c] = fma(-C[i * k + j], C[c * k + j], C[i * k + c]);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < k * k; e += SM_T) {
    const int i = e / k, j = e % k;
    T[e] = j <= i ? C[e] : 0.0;
  }
  for (int i = threadIdx.x; i < k; i += SM_T) {
    Tx[i] = dsc[i];
    Tx[LMAX + i] = invd[i];
  }
  if (threadIdx.x == 0) Tx[2 * LMAX] = 1.0;
  return true;
}

__device__ __forceinline__ void eig_orth_body(const double* __restrict__ G, int k, double tau,
                                              double* T, double* Tx, int* kept, int* err,
                                              double* smd) {
  const int Np = k + (k & 1);
  double* A = smd;
  double* V = A + (size_t)Np * k;
  double* nrm = V + (size_t)Np * Np;
  int* ord = reinterpret_cast<int*>(nrm + Np + (size_t)Np * Np);
  if (chol_orth(G, k, tau, A, nrm, T, Tx)) {
    if (threadIdx.x == 0) *kept = k;
    return;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < Np * k; e += SM_T) {
    int c = e / k, i = e % k;
    A[e] = c < k ? G[i * k + c] : 0.0;
  }
  set_identity(V, Np);
  __syncthreads();
  int sw = jacobi_osvd<double>(A, k, Np, V, JAC_MAX_SWEEPS);
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
    Tx[2 * LMAX] = 0.0;   // T is the map itself
    if (sw > JAC_MAX_SWEEPS - 1) atomicOr(err, ERR_NOTCONV);
  }
}

__global__ void __launch_bounds__(SM_T)
eig_orth_kernel(const double* __restrict__ G, int k, double tau, double* T, double* Tx, int* kept,
                int* err) {
  extern __shared__ double smd[];
  eig_orth_body(G, k, tau, T, Tx, kept, err, smd);
}

// One CTA per problem: problem b's transform on block b, the same arithmetic
// as its own eig_orth_kernel launch.
__global__ void __launch_bounds__(SM_T) eig_orth_group_kernel(const EigOrthProb* __restrict__ probs) {
  extern __shared__ double smd[];
  const EigOrthProb q = probs[blockIdx.x];
  eig_orth_body(q.G, q.k, q.tau, q.T, q.Tx, q.kept, q.err, smd);
}

void launch_eig_orth(const double* G, int k, double tau, double* T, double* Tx, int* kept, int* err,
                     cudaStream_t s) {
  note_launch(1);
  int Np = k + (k & 1);
  size_t smem = small_smem(k, Np);
  cudaFuncSetAttribute(eig_orth_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  eig_orth_kernel<<<1, SM_T, smem, s>>>(G, k, tau, T, Tx, kept, err);
}

void launch_eig_orth_group(const EigOrthProb* probs, int count, int max_k, cudaStream_t s) {
  if (count < 1) return;
  note_launch(1);
  const int Np = max_k + (max_k & 1);
  const size_t smem = small_smem(max_k, Np);
  cudaFuncSetAttribute(eig_orth_group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  eig_orth_group_kernel<<<count, SM_T, smem, s>>>(probs);
}

// ------------------------------------------------------ Rayleigh-Ritz SVD
// P = Q2^T Bt (k2 x k1, row-major).  The Rayleigh-Ritz matrix is
// B = Q^T X = P^T Q2^T, and P^T (k1 x k2) = Ut S Wt^T.  Column c of P^T is
// row c of P, so P's memory is P^T in column-major order.
// fp32_only (the forms with FP32 factors, whose range-finder bases and P are
// FP32-accurate): the FP32 sweeps alone, their A and V taken to FP64.
__device__ __forceinline__ void rr_svd_body(const double* __restrict__ P, int k2, int k1,
                                            double* sigma, double* Ut, double* Wt, int fp32_only,
                                            int* err, double* smd) {
  const int Np = k2 + (k2 & 1);
  double* A = smd;                  // Np columns x k1 rows
  double* V = A + (size_t)Np * k1;  // Np x Np
  double* nrm = V + (size_t)Np * Np;
  double* T = nrm + Np;                                        // Np x k1 (k1 <= Np)
  int* ord = reinterpret_cast<int*>(nrm + Np + (size_t)Np * Np);
  float* A32 = reinterpret_cast<float*>(ord + Np);            // Np x k1
  float* V32 = A32 + (size_t)Np * k1;                          // Np x Np
  for (int e = threadIdx.x; e < Np * k1; e += SM_T) {
    int c = e / k1, i = e % k1;
    A[e] = c < k2 ? P[(size_t)c * k1 + i] : 0.0;
  }
  __syncthreads();
  int sw;
  if (fp32_only) {
    for (int e = threadIdx.x; e < Np * k1; e += SM_T) A32[e] = (float)A[e];
    for (int e = threadIdx.x; e < Np * Np; e += SM_T) V32[e] = (e / Np == e % Np) ? 1.f : 0.f;
    __syncthreads();
    sw = jacobi_osvd_f32(A32, k1, Np, V32, JAC_MAX_SWEEPS);
    for (int e = threadIdx.x; e < Np * k1; e += SM_T) A[e] = (double)A32[e];
    for (int e = threadIdx.x; e < Np * Np; e += SM_T) V[e] = (double)V32[e];
    __syncthreads();
  } else {
    sw = jacobi_osvd_mixed(A, k1, Np, V, A32, V32, T);
  }
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

__global__ void __launch_bounds__(SM_T)
rr_svd_kernel(const double* __restrict__ P, int k2, int k1, double* sigma, double* Ut, double* Wt,
              int fp32_only, int* err) {
  extern __shared__ double smd[];
  rr_svd_body(P, k2, k1, sigma, Ut, Wt, fp32_only, err, smd);
}

// One CTA per problem: problem b's SVD on block b, the same arithmetic as its
// own rr_svd_kernel launch.
__global__ void __launch_bounds__(SM_T) rr_svd_group_kernel(const RrSvdProb* __restrict__ probs) {
  extern __shared__ double smd[];
  const RrSvdProb q = probs[blockIdx.x];
  rr_svd_body(q.P, q.k2, q.k1, q.sigma, q.Ut, q.Wt, q.fp32_only, q.err, smd);
}

static size_t rr_svd_smem(int k2, int k1) {
  const int Np = k2 + (k2 & 1);
  // FP64 panels plus the FP32 copies of the mixed-precision Jacobi
  return small_smem(k1 > Np ? k1 : Np, Np) + sizeof(float) * ((size_t)Np * k1 + (size_t)Np * Np);
}

void launch_rr_svd(const double* P, int k2, int k1, double* sigma, double* Ut, double* Wt,
                   int fp32_only, int* err, cudaStream_t s) {
  note_launch(1);
  const size_t smem = rr_svd_smem(k2, k1);
  cudaFuncSetAttribute(rr_svd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  rr_svd_kernel<<<1, SM_T, smem, s>>>(P, k2, k1, sigma, Ut, Wt, fp32_only, err);
}

void launch_rr_svd_group(const RrSvdProb* probs, int count, int max_k2, int max_k1,
                         cudaStream_t s) {
  if (count < 1) return;
  note_launch(1);
  const size_t smem = rr_svd_smem(max_k2, max_k1);
  cudaFuncSetAttribute(rr_svd_group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  rr_svd_group_kernel<<<count, SM_T, smem, s>>>(probs);
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
  note_launch(1);
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
  note_launch(1);
  svd_finish_kernel<<<1, 256, 0, s>>>(sigma, Ut, Wt, k1, k2, r, colsumQ, colsumQ2, Tu, Tv,
                                      sigma_out);
}

// ------------------------------------------------- equivalence tools (App. F, H)
// Generalized orthogonal transform between two factorisations (App. F): from
// G = U_e^T U_e and C = U_e^T U_alg (k x k, FP64), Z = G^-1 C -- the
// least-squares map from U_e to U_alg, Q Gamma^-1 P^T U_alg for the thin SVD
// U_e = P Gamma Q^T -- by a Cholesky factorisation of G, then Z = R1 Lambda
// R2^T by one-sided Jacobi (Lambda descending) and Zit = R1 Lambda^-1 R2^T,
// the map of the V factors.  Row-major outputs; ERR_NOTCONV when G is not
// positive definite or Jacobi did not converge.
__global__ void __launch_bounds__(SM_T)
equiv_svd_kernel(const double* __restrict__ Gg, const double* __restrict__ Cg, int k, double* R1,
                 double* lam, double* R2, double* Zout, double* Zit, int* err) {
  extern __shared__ double smd[];
  const int Np = k + (k & 1);
  double* L = smd;                    // k x k, Cholesky factor (lower), row-major
  double* Z = L + (size_t)k * k;      // k x k, C then Z (row-major)
  double* A = Z + (size_t)k * k;      // Np columns x k rows (column-major)
  double* V = A + (size_t)Np * k;     // Np x Np
  double* nrm = V + (size_t)Np * Np;
  int* ord = reinterpret_cast<int*>(nrm + Np);
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  for (int e = threadIdx.x; e < k * k; e += SM_T) {
    L[e] = Gg[e];
    Z[e] = Cg[e];
  }
  __syncthreads();
  // Cholesky, right-looking: column j, then the trailing update
  for (int j = 0; j < k; ++j) {
    if (threadIdx.x == 0) {
      const double d = L[j * k + j];
      if (!(d > 0.0)) bad = 1;
      L[j * k + j] = d > 0.0 ? sqrt(d) : 1.0;
    }
    __syncthreads();
    const double ljj = L[j * k + j];
    for (int i = j + 1 + threadIdx.x; i < k; i += SM_T) L[i * k + j] /= ljj;
    __syncthreads();
    for (int e = threadIdx.x; e < (k - j - 1) * (k - j - 1); e += SM_T) {
      const int i = j + 1 + e / (k - j - 1), c = j + 1 + e % (k - j - 1);
      if (c <= i) L[i * k + c] = fma(-L[i * k + j], L[c * k + j], L[i * k + c]);
    }
    __syncthreads();
  }
  // Z = L^-T L^-1 C, one right-hand side column per thread
  for (int c = threadIdx.x; c < k; c += SM_T) {
    for (int i = 0; i < k; ++i) {           // forward: L y = C_:c
      double sacc = Z[i * k + c];
      for (int p = 0; p < i; ++p) sacc = fma(-L[i * k + p], Z[p * k + c], sacc);
      Z[i * k + c] = sacc / L[i * k + i];
    }
    for (int i = k - 1; i >= 0; --i) {      // backward: L^T z = y
      double sacc = Z[i * k + c];
      for (int p = i + 1; p < k; ++p) sacc = fma(-L[p * k + i], Z[p * k + c], sacc);
      Z[i * k + c] = sacc / L[i * k + i];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < Np * k; e += SM_T) {
    const int c = e / k, i = e % k;
    A[e] = c < k ? Z[i * k + c] : 0.0;
  }
  set_identity(V, Np);
  __syncthreads();
  const int sw = jacobi_osvd<double>(A, k, Np, V, JAC_MAX_SWEEPS);
  sort_desc(A, k, Np, nrm, ord);
  for (int e = threadIdx.x; e < k * k; e += SM_T) {
    const int i = e / k, j = e % k;
    const int c = ord[j];
    R1[e] = nrm[c] > 0.0 ? A[(size_t)c * k + i] / nrm[c] : 0.0;
    R2[e] = V[(size_t)c * Np + i];
    if (Zout) Zout[e] = Z[e];
  }
  for (int j = threadIdx.x; j < k; j += SM_T) lam[j] = nrm[ord[j]];
  __syncthreads();
  // Zit = R1 Lambda^-1 R2^T = sum_j (a_j / s_j^2) v_j^T over the columns
  for (int e = threadIdx.x; e < k * k; e += SM_T) {
    const int i = e / k, p = e % k;
    double sacc = 0.0;
    for (int j = 0; j < k; ++j) {
      const int c = ord[j];
      const double s2 = nrm[c] * nrm[c];
      if (s2 > 0.0) sacc = fma(A[(size_t)c * k + i] / s2, V[(size_t)c * Np + p], sacc);
    }
    Zit[e] = sacc;
  }
  if (threadIdx.x == 0 && (bad || sw > JAC_MAX_SWEEPS - 1)) atomicOr(err, ERR_NOTCONV);
}

void launch_equiv_svd(const double* G, const double* C, int k, double* R1, double* lam, double* R2,
                      double* Z, double* Zit, int* err, cudaStream_t s) {
  note_launch(1);
  const int Np = k + (k & 1);
  const size_t smem = sizeof(double) * (2 * (size_t)k * k + (size_t)Np * k + (size_t)Np * Np + Np) +
                      sizeof(int) * Np + 64;
  cudaFuncSetAttribute(equiv_svd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  equiv_svd_kernel<<<1, SM_T, smem, s>>>(G, C, k, R1, lam, R2, Z, Zit, err);
}

// Permutation check of App. H from the Grams GAA = U_A^T U_A, GBB = U_B^T U_B
// and GAB = U_A^T U_B (k x k, FP64).  Cosines cos_ij = G_ij / sqrt(G_ii G_jj)
// (0 for a zero column).  Step 1: pairs (i, j) taken one to one in decreasing
// cos(U_A^(i), U_B^(j)) (ties by lower i, then lower j) while the cosine is
// >= 1 - eps.  Step 2: on the candidates (ordered by i), the columns of the
// self- and cross-similarity matrices M, N, S sorted descending and rounded to
// one decimal (floor(10 x + 1/2)); candidate c stays when M's column c equals
// N's and S's at more than keep_frac of its positions.  Output: b_of_a[i] =
// the matched column of U_B, or -1; *count = pairs kept.
constexpr int PC_T = 256;

__device__ __forceinline__ double cos_of(const double* G, int ldg, int i, int j, const double* na,
                                         const double* nb) {
  const double den = na[i] * nb[j];
  return den > 0.0 ? G[i * ldg + j] / den : 0.0;
}

__global__ void __launch_bounds__(PC_T)
perm_check_kernel(const double* __restrict__ GAA, const double* __restrict__ GBB,
                  const double* __restrict__ GAB, int k, double eps, double keep_frac,
                  int* b_of_a, int* count) {
  __shared__ double na[RMAX], nb[RMAX];
  __shared__ double S0[RMAX * RMAX];
  __shared__ unsigned char used_a[RMAX], used_b[RMAX];
  __shared__ int pa[RMAX], pb[RMAX], npair, stop;
  __shared__ double bv[PC_T];
  __shared__ int bi[PC_T];
  __shared__ int keep[RMAX];
  const int t = threadIdx.x;
  for (int i = t; i < k; i += PC_T) {
    na[i] = sqrt(fmax(GAA[i * k + i], 0.0));
    nb[i] = sqrt(fmax(GBB[i * k + i], 0.0));
    used_a[i] = 0;
    used_b[i] = 0;
  }
  if (t == 0) {
    npair = 0;
    stop = 0;
  }
  __syncthreads();
  for (int e = t; e < k * k; e += PC_T) S0[e] = cos_of(GAB, k, e / k, e % k, na, nb);
  __syncthreads();
  // step 1: greedy one-to-one pairing
  for (int round = 0; round < k; ++round) {
    double best = -INFINITY;
    int bidx = -1;
    for (int e = t; e < k * k; e += PC_T) {
      const int i = e / k, j = e % k;
      if (used_a[i] || used_b[j]) continue;
      const double v = S0[e];
      if (v > best || (v == best && (bidx < 0 || e < bidx))) {   // e = i k + j: (i, j) order
        best = v;
        bidx = e;
      }
    }
    bv[t] = best;
    bi[t] = bidx;
    __syncthreads();
    for (int w = PC_T / 2; w > 0; w >>= 1) {
      if (t < w) {
        const double v2 = bv[t + w];
        const int i2 = bi[t + w];
        if (i2 >= 0 && (bi[t] < 0 || v2 > bv[t] || (v2 == bv[t] && i2 < bi[t]))) {
          bv[t] = v2;
          bi[t] = i2;
        }
      }
      __syncthreads();
    }
    if (t == 0) {
      if (bi[0] < 0 || bv[0] < 1.0 - eps) {
        stop = 1;
      } else {
        const int i = bi[0] / k, j = bi[0] % k;
        used_a[i] = 1;
        used_b[j] = 1;
        pa[npair] = i;
        pb[npair] = j;
        ++npair;
      }
    }
    __syncthreads();
    if (stop) break;
  }
  // candidates in increasing index of U_A
  if (t == 0) {
    for (int x = 1; x < npair; ++x)
      for (int y = x; y > 0 && pa[y - 1] > pa[y]; --y) {
        int q = pa[y]; pa[y] = pa[y - 1]; pa[y - 1] = q;
        q = pb[y]; pb[y] = pb[y - 1]; pb[y - 1] = q;
      }
  }
  __syncthreads();
  const int nc = npair;
  // step 2: one thread per candidate column; the column's entries sorted by
  // rank (descending value, ties by position) and compared after rounding
  for (int c = t; c < nc; c += PC_T) {
    double srt[3][RMAX];
    for (int which = 0; which < 3; ++which) {
      for (int x = 0; x < nc; ++x) {
        double vx;
        if (which == 0) vx = cos_of(GAA, k, pa[x], pa[c], na, na);
        else if (which == 1) vx = cos_of(GBB, k, pb[x], pb[c], nb, nb);
        else vx = cos_of(GAB, k, pa[x], pb[c], na, nb);
        int rank = 0;
        for (int y = 0; y < nc; ++y) {
          double vy;
          if (which == 0) vy = cos_of(GAA, k, pa[y], pa[c], na, na);
          else if (which == 1) vy = cos_of(GBB, k, pb[y], pb[c], nb, nb);
          else vy = cos_of(GAB, k, pa[y], pb[c], na, nb);
          if (vy > vx || (vy == vx && y < x)) ++rank;
        }
        srt[which][rank] = vx;
      }
    }
    int match = 0;
    for (int pos = 0; pos < nc; ++pos) {
      const double km = floor(10.0 * srt[0][pos] + 0.5), kn = floor(10.0 * srt[1][pos] + 0.5),
                   ks = floor(10.0 * srt[2][pos] + 0.5);
      if (km == kn && km == ks) ++match;
    }
    keep[c] = (double)match / (double)nc > keep_frac ? 1 : 0;
  }
  __syncthreads();
  for (int i = t; i < k; i += PC_T) b_of_a[i] = -1;
  __syncthreads();
  if (t == 0) {
    int kept = 0;
    for (int c = 0; c < nc; ++c)
      if (keep[c]) {
        b_of_a[pa[c]] = pb[c];
        ++kept;
      }
    *count = kept;
  }
}

void launch_perm_check(const double* GAA, const double* GBB, const double* GAB, int k, double eps,
                       double keep_frac, int* b_of_a, int* count, cudaStream_t s) {
  note_launch(1);
  perm_check_kernel<<<1, PC_T, 0, s>>>(GAA, GBB, GAB, k, eps, keep_frac, b_of_a, count);
}

}  // namespace enmf
