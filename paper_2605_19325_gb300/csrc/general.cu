// Algorithm 4 (App. A.2): ADMM for the generalized rotation of Eq. 5,
//     minimise sum h(U* R1 Lambda R2) + sum h(V* R1 Lambda^-1 R2)
// over orthogonal R1, R2 and diagonal Lambda > 0, with the splitting
// W1 = W_svd R1, W2 = [W11 Lambda; W12 Lambda^-1], W3 = W2 R2 and the scaled
// duals M, N, P.  Per step, in the order of Algorithm 4:
//   pass A (rows)   W3 = prox_t(W2 R2 - P)            (the Eq. 7 form)
//                   W1 from its closed form (per column, with lambda_j)
//                   block partials of W_svd^T (W1 + M)
//   R1 = polar(...)                                     (small.cu)
//   pass B (rows)   W2 from its closed form, block partials of W2^T (W3 + P)
//                   and of the four column sums of the Lambda quartic
//   R2 = polar(...), lambda_i = the positive root of
//        a l^4 - b l^3 + c l - d = 0 with the least objective   (one thread each)
//   pass C (rows)   M += W1 - W_svd R1, N += W2 - [W11 Lambda; W12 Lambda^-1],
//                   P += W3 - W2 R2
// The rows are independent (one thread per row, the r x r operands in shared
// memory); the reductions are FP64 block partials summed in block order.
#include <vector>

#include "internal.h"

namespace enmf {
namespace {

constexpr int GR_T = 64;   // threads (rows) per block

// per-block FP64 partials of A^T B over the block's rows, A and B staged in
// shared memory as GR_T x k tiles; thread t owns entries t, t + GR_T, ...
__device__ __forceinline__ void tile_gram(const double* As, const double* Bs, int nr, int k,
                                          double* acc) {
  for (int q = 0; q * GR_T + (int)threadIdx.x < k * k; ++q) {
    const int e = q * GR_T + threadIdx.x;
    const int i = e / k, j = e % k;
    double s = acc[q];
    for (int rr = 0; rr < nr; ++rr) s = fma(As[rr * RMAX + i], Bs[rr * RMAX + j], s);
    acc[q] = s;
  }
}

constexpr int GQ = (RMAX * RMAX + GR_T - 1) / GR_T;   // Gram entries per thread

struct GenArgs {
  const void* Us;
  const void* Vs;
  void* W1;
  void* W2;
  void* W3;
  void* M;
  void* N;
  void* P;
  const double* R1;
  const double* R2;
  const double* lam;
  int64_t m, n;
  int k;
  double rho, gamma, t;
  double* part;    // NPART x (k * k + 4 RMAX)
  const int* done; // set once the stopping rule holds: every later kernel of the loop returns
};

template <typename TF>
__device__ __forceinline__ const TF* ws_row(const GenArgs& g, int64_t i) {
  return i < g.m ? (const TF*)g.Us + i * g.k : (const TF*)g.Vs + (i - g.m) * g.k;
}

// pass A
template <typename TF>
__global__ void __launch_bounds__(GR_T) gen_pass_a(GenArgs g) {
  if (*(volatile const int*)g.done) return;
  extern __shared__ double gsm[];
  const int k = g.k;
  double* R1s = gsm;                 // k x k
  double* R2s = R1s + k * k;         // k x k
  double* ls = R2s + k * k;          // RMAX
  double* As = ls + RMAX;            // GR_T x RMAX
  double* Bs = As + GR_T * RMAX;     // GR_T x RMAX
  for (int e = threadIdx.x; e < k * k; e += GR_T) {
    R1s[e] = g.R1[e];
    R2s[e] = g.R2[e];
  }
  for (int j = threadIdx.x; j < k; j += GR_T) ls[j] = g.lam[j];
  __syncthreads();
  const int64_t rows = g.m + g.n;
  const int64_t chunk = (rows + NPART - 1) / NPART;
  const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(rows, r0 + chunk);
  double acc[GQ];
#pragma unroll
  for (int q = 0; q < GQ; ++q) acc[q] = 0.0;
  const double inv_t = 1.0 / g.t;
  for (int64_t t0 = r0; t0 < r1; t0 += GR_T) {
    const int nr = (int)min((int64_t)GR_T, r1 - t0);
    const int64_t i = t0 + threadIdx.x;
    if (threadIdx.x < nr) {
      const TF* ws = ws_row<TF>(g, i);
      TF* w1 = (TF*)g.W1 + i * k;
      const TF* w2 = (const TF*)g.W2 + i * k;
      TF* w3 = (TF*)g.W3 + i * k;
      const TF* mr = (const TF*)g.M + i * k;
      const TF* nrw = (const TF*)g.N + i * k;
      const TF* pr = (const TF*)g.P + i * k;
      const bool ublk = i < g.m;
      for (int j = 0; j < k; ++j) {
        // W3 = prox(W2 R2 - P): entrywise minimiser of h(z) + t/2 (z - b)^2
        double b = -(double)pr[j];
        double wr1 = 0.0;
        for (int l = 0; l < k; ++l) {
          b = fma((double)w2[l], R2s[l * k + j], b);
          wr1 = fma((double)ws[l], R1s[l * k + j], wr1);
        }
        const double z = b > 0.0 ? b : (b >= -inv_t ? 0.0 : b + inv_t);
        w3[j] = (TF)z;
        // W1 closed form (column j, lambda_j)
        const double lj = ls[j];
        double v;
        if (ublk)
          v = (g.rho * (wr1 - (double)mr[j]) + g.gamma * lj * ((double)w2[j] + (double)nrw[j])) /
              (g.rho + g.gamma * lj * lj);
        else
          v = (g.rho * (wr1 - (double)mr[j]) + (g.gamma / lj) * ((double)w2[j] + (double)nrw[j])) /
              (g.rho + g.gamma / (lj * lj));
        w1[j] = (TF)v;
        As[threadIdx.x * RMAX + j] = (double)ws[j];
        Bs[threadIdx.x * RMAX + j] = (double)(TF)v + (double)mr[j];
      }
    }
    __syncthreads();
    tile_gram(As, Bs, nr, k, acc);
    __syncthreads();
  }
  double* part = g.part + (int64_t)blockIdx.x * (k * k + 4 * RMAX);
#pragma unroll
  for (int q = 0; q < GQ; ++q) {
    const int e = q * GR_T + threadIdx.x;
    if (e < k * k) part[e] = acc[q];
  }
}

// pass B
template <typename TF>
__global__ void __launch_bounds__(GR_T) gen_pass_b(GenArgs g) {
  if (*(volatile const int*)g.done) return;
  extern __shared__ double gsm[];
  const int k = g.k;
  double* R2s = gsm;                 // k x k
  double* ls = R2s + k * k;          // RMAX
  double* As = ls + RMAX;            // GR_T x RMAX
  double* Bs = As + GR_T * RMAX;     // GR_T x RMAX
  double (*cs)[RMAX] = reinterpret_cast<double (*)[RMAX]>(Bs + GR_T * RMAX);   // 4 x RMAX
  for (int e = threadIdx.x; e < k * k; e += GR_T) R2s[e] = g.R2[e];
  for (int j = threadIdx.x; j < k; j += GR_T) ls[j] = g.lam[j];
  for (int e = threadIdx.x; e < 4 * RMAX; e += GR_T) cs[e / RMAX][e % RMAX] = 0.0;
  __syncthreads();
  const int64_t rows = g.m + g.n;
  const int64_t chunk = (rows + NPART - 1) / NPART;
  const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(rows, r0 + chunk);
  double acc[GQ];
#pragma unroll
  for (int q = 0; q < GQ; ++q) acc[q] = 0.0;
  const double den = g.gamma + g.t;
  for (int64_t t0 = r0; t0 < r1; t0 += GR_T) {
    const int nr = (int)min((int64_t)GR_T, r1 - t0);
    const int64_t i = t0 + threadIdx.x;
    if (threadIdx.x < nr) {
      const TF* w1 = (const TF*)g.W1 + i * k;
      TF* w2 = (TF*)g.W2 + i * k;
      const TF* w3 = (const TF*)g.W3 + i * k;
      const TF* nrw = (const TF*)g.N + i * k;
      const TF* pr = (const TF*)g.P + i * k;
      const bool ublk = i < g.m;
      for (int j = 0; j < k; ++j) {
        // (W3 + P) R2^T, column j: sum_l (w3 + p)_l R2[j][l]
        double q = 0.0;
        for (int l = 0; l < k; ++l) q = fma((double)w3[l] + (double)pr[l], R2s[j * k + l], q);
        const double lj = ls[j];
        const double sc = ublk ? lj : 1.0 / lj;
        const double v = (g.gamma * (double)w1[j] * sc - g.gamma * (double)nrw[j] + g.t * q) / den;
        w2[j] = (TF)v;
        As[threadIdx.x * RMAX + j] = (double)(TF)v;
        Bs[threadIdx.x * RMAX + j] = (double)w3[j] + (double)pr[j];
      }
    }
    __syncthreads();
    tile_gram(As, Bs, nr, k, acc);
    // the quartic's column sums: over the U block a = |W11|^2, b = (W21 + N1).W11;
    // over the V block c = (W22 + N2).W12, d = |W12|^2 (thread j sums column j
    // over the tile's rows, in row order)
    for (int j = threadIdx.x; j < k; j += GR_T) {
      double a = cs[0][j], b = cs[1][j], c = cs[2][j], d = cs[3][j];
      for (int rr = 0; rr < nr; ++rr) {
        const int64_t ii = t0 + rr;
        const double x1 = (double)((const TF*)g.W1)[ii * k + j];
        const double x2n = As[rr * RMAX + j] + (double)((const TF*)g.N)[ii * k + j];
        if (ii < g.m) {
          a = fma(x1, x1, a);
          b = fma(x2n, x1, b);
        } else {
          c = fma(x2n, x1, c);
          d = fma(x1, x1, d);
        }
      }
      cs[0][j] = a;
      cs[1][j] = b;
      cs[2][j] = c;
      cs[3][j] = d;
    }
    __syncthreads();
  }
  double* part = g.part + (int64_t)blockIdx.x * (k * k + 4 * RMAX);
#pragma unroll
  for (int q = 0; q < GQ; ++q) {
    const int e = q * GR_T + threadIdx.x;
    if (e < k * k) part[e] = acc[q];
  }
  for (int e = threadIdx.x; e < 4 * RMAX; e += GR_T) part[k * k + e] = cs[e / RMAX][e % RMAX];
}

// pass C: the dual updates with the new R1, Lambda, R2
template <typename TF>
__global__ void __launch_bounds__(GR_T) gen_pass_c(GenArgs g) {
  if (*(volatile const int*)g.done) return;
  extern __shared__ double gsm[];
  const int k = g.k;
  double* R1s = gsm;
  double* R2s = R1s + k * k;
  double* ls = R2s + k * k;
  for (int e = threadIdx.x; e < k * k; e += GR_T) {
    R1s[e] = g.R1[e];
    R2s[e] = g.R2[e];
  }
  for (int j = threadIdx.x; j < k; j += GR_T) ls[j] = g.lam[j];
  __syncthreads();
  const int64_t rows = g.m + g.n;
  for (int64_t i = (int64_t)blockIdx.x * GR_T + threadIdx.x; i < rows;
       i += (int64_t)gridDim.x * GR_T) {
    const TF* ws = ws_row<TF>(g, i);
    const TF* w1 = (const TF*)g.W1 + i * k;
    const TF* w2 = (const TF*)g.W2 + i * k;
    const TF* w3 = (const TF*)g.W3 + i * k;
    TF* mr = (TF*)g.M + i * k;
    TF* nrw = (TF*)g.N + i * k;
    TF* pr = (TF*)g.P + i * k;
    const bool ublk = i < g.m;
    for (int j = 0; j < k; ++j) {
      double wr1 = 0.0, w2r2 = 0.0;
      for (int l = 0; l < k; ++l) {
        wr1 = fma((double)ws[l], R1s[l * k + j], wr1);
        w2r2 = fma((double)w2[l], R2s[l * k + j], w2r2);
      }
      mr[j] = (TF)((double)mr[j] + (double)w1[j] - wr1);
      const double sc = ublk ? ls[j] : 1.0 / ls[j];
      nrw[j] = (TF)((double)nrw[j] + (double)w2[j] - (double)w1[j] * sc);
      pr[j] = (TF)((double)pr[j] + (double)w3[j] - w2r2);
    }
  }
}

// Sum of the NPART block partials of width w into out, in block order.
__global__ void gen_reduce(const double* __restrict__ part, int stride, int off, int w,
                           double* __restrict__ out, const int* done) {
  if (*(volatile const int*)done) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < w; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < NPART; ++b) s += part[(int64_t)b * stride + off + e];
    out[e] = s;
  }
}

// p(l) = a l^4 - b l^3 + c l - d and the objective (up to a constant)
// g(l) = a l^2 - 2 b l + d / l^2 - 2 c / l.
__device__ __forceinline__ double qp(double a, double b, double c, double d, double l) {
  return (((a * l - b) * l) * l + c) * l - d;
}
__device__ __forceinline__ double qg(double a, double b, double c, double d, double l) {
  return a * l * l - 2.0 * b * l + d / (l * l) - 2.0 * c / l;
}

// The root of f in [lo, hi] by bisection to the last bit (f(lo), f(hi) of
// opposite signs or zero).
template <typename F>
__device__ double bisect(F f, double lo, double hi) {
  double flo = f(lo);
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (!(mid > lo && mid < hi)) break;
    const double fm = f(mid);
    if (fm == 0.0) return mid;
    if ((fm < 0.0) == (flo < 0.0)) {
      lo = mid;
      flo = fm;
    } else {
      hi = mid;
    }
  }
  return 0.5 * (lo + hi);
}

// Lambda update (one thread per column) and the step's change
// |R1n - R1| + |R2n - R2| + |lam_new - lam| (Frobenius norms) into *change;
// R1 <- R1n, R2 <- R2n.  sums: the quartic coefficients (4 x RMAX).  The
// positive real roots of p are separated by the positive critical points of
// p (roots of p' = 4 a l^3 - 3 b l^2 + c, whose own critical points are 0 and
// b / 2a): every interval between consecutive points of {0, those roots, an
// upper bound of the roots} holds at most one root, found by bisection; the
// root with the least g wins (the previous lambda when there is none).
__global__ void gen_lambda_kernel(const double* __restrict__ sums, int k, double* lam,
                                  double* R1, const double* R1n, double* R2, const double* R2n,
                                  double* change, int* done, int* steps, double thr) {
  __shared__ double red[RMAX];
  __shared__ double dl[RMAX];
  if (*(volatile int*)done) return;
  const int j = threadIdx.x;
  double dlam2 = 0.0;
  if (j < k) {
    const double a = sums[0 * RMAX + j], b = sums[1 * RMAX + j], c = sums[2 * RMAX + j],
                 d = sums[3 * RMAX + j];
    const double prev = lam[j];
    double best = prev;
    if (a > 0.0 && d > 0.0) {
      // upper bound of the positive roots (Cauchy): 1 + max(|b|, |c|, |d|) / a
      const double ub = 1.0 + fmax(fabs(b), fmax(fabs(c), d)) / a;
      // critical points of p in (0, ub): roots of p' on (0, lc) and (lc, ub)
      const double lc = b > 0.0 ? b / (2.0 * a) : 0.0;
      auto dp = [&](double l) { return (4.0 * a * l - 3.0 * b) * l * l + c; };
      double pts[5];
      int np = 0;
      pts[np++] = 0.0;
      if (lc > 0.0 && lc < ub) {
        if ((dp(0.0) > 0.0) != (dp(lc) > 0.0)) pts[np++] = bisect(dp, 0.0, lc);
        if ((dp(lc) > 0.0) != (dp(ub) > 0.0)) pts[np++] = bisect(dp, lc, ub);
      } else if ((dp(0.0) > 0.0) != (dp(ub) > 0.0)) {
        pts[np++] = bisect(dp, 0.0, ub);
      }
      pts[np++] = ub;
      auto pf = [&](double l) { return qp(a, b, c, d, l); };
      double gbest = INFINITY;
      bool found = false;
      for (int q = 0; q + 1 < np; ++q) {
        const double lo = pts[q], hi = pts[q + 1];
        const double plo = pf(lo), phi = pf(hi);
        if (plo == 0.0 && lo > 0.0) {
          const double gv = qg(a, b, c, d, lo);
          if (gv < gbest) { gbest = gv; best = lo; found = true; }
        }
        if ((plo < 0.0 && phi > 0.0) || (plo > 0.0 && phi < 0.0)) {
          const double rt = bisect(pf, lo, hi);
          if (rt > 0.0) {
            const double gv = qg(a, b, c, d, rt);
            if (gv < gbest) { gbest = gv; best = rt; found = true; }
          }
        }
      }
      if (!found) best = prev;
    }
    dlam2 = (best - prev) * (best - prev);
    dl[j] = best;
  }
  __syncthreads();
  double d2 = dlam2;
  double r1 = 0.0, r2 = 0.0;
  for (int e = j; e < k * k; e += blockDim.x) {
    r1 = fma(R1n[e] - R1[e], R1n[e] - R1[e], r1);
    r2 = fma(R2n[e] - R2[e], R2n[e] - R2[e], r2);
  }
  // three fixed-order block sums (blockDim = RMAX threads)
  double out[3] = {0.0, 0.0, 0.0};
  const double in[3] = {d2, r1, r2};
  for (int q = 0; q < 3; ++q) {
    red[j] = in[q];
    __syncthreads();
    for (int s = RMAX / 2; s > 0; s >>= 1) {
      if (j < s) red[j] += red[j + s];
      __syncthreads();
    }
    out[q] = red[0];
    __syncthreads();
  }
  for (int e = j; e < k * k; e += blockDim.x) {
    R1[e] = R1n[e];
    R2[e] = R2n[e];
  }
  if (j < k) lam[j] = dl[j];
  if (j == 0) {
    const double ch = sqrt(out[1]) + sqrt(out[2]) + sqrt(out[0]);
    *change = ch;
    *steps += 1;
    if (ch <= thr) *done = 1;   // the next kernels of the loop return at once
  }
}

// U <- U R1 Lambda R2 (V: R1 Lambda^-1 R2) in place, row by row.
template <typename TF>
__global__ void __launch_bounds__(GR_T) gen_apply(TF* F, int64_t rows, int k, const double* R1,
                                                  const double* lam, const double* R2, int inv) {
  __shared__ double T[RMAX * RMAX];
  for (int e = threadIdx.x; e < k * k; e += GR_T) {
    const int i = e / k, j = e % k;
    double s = 0.0;
    for (int l = 0; l < k; ++l) {
      const double sc = inv ? 1.0 / lam[l] : lam[l];
      s = fma(R1[i * k + l] * sc, R2[l * k + j], s);
    }
    T[e] = s;
  }
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * GR_T + threadIdx.x; i < rows;
       i += (int64_t)gridDim.x * GR_T) {
    double x[RMAX];
    for (int l = 0; l < k; ++l) x[l] = (double)F[i * k + l];
    for (int j = 0; j < k; ++j) {
      double s = 0.0;
      for (int l = 0; l < k; ++l) s = fma(x[l], T[l * k + j], s);
      F[i * k + j] = (TF)s;
    }
  }
}

template <typename TF>
void pass(int which, const GenArgs& g, cudaStream_t s) {
  note_launch(1);
  const int k = g.k;
  if (which == 0) {
    const size_t sm = sizeof(double) * (2 * (size_t)k * k + RMAX + 2 * (size_t)GR_T * RMAX);
    cudaFuncSetAttribute(gen_pass_a<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    gen_pass_a<TF><<<NPART, GR_T, sm, s>>>(g);
  } else if (which == 1) {
    const size_t sm = sizeof(double) * ((size_t)k * k + RMAX + 2 * (size_t)GR_T * RMAX + 4 * RMAX);
    cudaFuncSetAttribute(gen_pass_b<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    gen_pass_b<TF><<<NPART, GR_T, sm, s>>>(g);
  } else {
    const size_t sm = sizeof(double) * (2 * (size_t)k * k + RMAX);
    cudaFuncSetAttribute(gen_pass_c<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const int64_t rows = g.m + g.n;
    int blocks = (int)min((int64_t)1024, (rows + GR_T - 1) / GR_T);
    gen_pass_c<TF><<<blocks < 1 ? 1 : blocks, GR_T, sm, s>>>(g);
  }
}

}  // namespace

// ---------------------------------------------------------------- host
// Workspace (device, FP64 unless noted): W1, W2, W3, M, N, P ((m + n) x k in
// the factor type), R1, R2, R1n, R2n, D1, D2 (LMAX^2), lam (RMAX), B (k x k),
// sums (4 RMAX), change, part (NPART x (k^2 + 4 RMAX)).
size_t general_ws_bytes(int64_t m, int64_t n, int k, int fdt) {
  const size_t fs = type_size(fdt);
  auto a = [](size_t b) { return (b + 255) & ~(size_t)255; };
  return 6 * a((size_t)(m + n) * k * fs) + 6 * a((size_t)LMAX * LMAX * 8) + a(RMAX * 8) +
         a((size_t)k * k * 8) + a(4 * RMAX * 8) + a(64) + a(64) +
         a((size_t)NPART * ((size_t)k * k + 4 * RMAX) * 8);
}

enmf_status run_general_rotation(const void* U, const void* V, int64_t m, int64_t n, int k,
                                 int fdt, void* ws, double rho, int max_iter, double tol,
                                 double* R1_out, double* lam_out, double* R2_out, int* err,
                                 int* steps_out, double* change_out, bool* converged,
                                 cudaStream_t s) {
  const size_t fs = type_size(fdt);
  auto a = [](size_t b) { return (b + 255) & ~(size_t)255; };
  char* p = (char*)ws;
  auto take = [&](size_t b) { void* q = p; p += a(b); return q; };
  const size_t wb = (size_t)(m + n) * k * fs;
  void* W1 = take(wb);
  void* W2 = take(wb);
  void* W3 = take(wb);
  void* M = take(wb);
  void* N = take(wb);
  void* P = take(wb);
  double* R1 = (double*)take(LMAX * LMAX * 8);
  double* R2 = (double*)take(LMAX * LMAX * 8);
  double* R1n = (double*)take(LMAX * LMAX * 8);
  double* R2n = (double*)take(LMAX * LMAX * 8);
  double* D1 = (double*)take(LMAX * LMAX * 8);
  double* D2 = (double*)take(LMAX * LMAX * 8);
  double* lam = (double*)take(RMAX * 8);
  double* Bm = (double*)take((size_t)k * k * 8);
  double* sums = (double*)take(4 * RMAX * 8);
  double* change = (double*)take(64);
  int* flags = (int*)take(64);   // [0] done, [1] steps
  double* part = (double*)take((size_t)NPART * ((size_t)k * k + 4 * RMAX) * 8);
  // start: R1 = R2 = I, Lambda = I, W1 = W2 = W3 = W_svd, zero duals,
  // identity warm starts of the two polar factors
  const int Np = k + (k & 1);
  std::vector<double> eye((size_t)k * k, 0.0), eyeD((size_t)Np * Np, 0.0), ones(k, 1.0);
  for (int i = 0; i < k; ++i) eye[(size_t)i * k + i] = 1.0;
  for (int i = 0; i < Np; ++i) eyeD[(size_t)i * Np + i] = 1.0;
  if (cudaMemcpyAsync(R1, eye.data(), eye.size() * 8, cudaMemcpyHostToDevice, s) ||
      cudaMemcpyAsync(R2, eye.data(), eye.size() * 8, cudaMemcpyHostToDevice, s) ||
      cudaMemcpyAsync(D1, eyeD.data(), eyeD.size() * 8, cudaMemcpyHostToDevice, s) ||
      cudaMemcpyAsync(D2, eyeD.data(), eyeD.size() * 8, cudaMemcpyHostToDevice, s) ||
      cudaMemcpyAsync(lam, ones.data(), (size_t)k * 8, cudaMemcpyHostToDevice, s))
    return ENMF_ECUDA;
  for (void* W : {W1, W2, W3}) {
    if (cudaMemcpyAsync(W, U, (size_t)m * k * fs, cudaMemcpyDeviceToDevice, s) ||
        cudaMemcpyAsync((char*)W + (size_t)m * k * fs, V, (size_t)n * k * fs,
                        cudaMemcpyDeviceToDevice, s))
      return ENMF_ECUDA;
  }
  for (void* D : {M, N, P})
    if (cudaMemsetAsync(D, 0, wb, s)) return ENMF_ECUDA;
  if (cudaMemsetAsync(flags, 0, 64, s) || cudaMemsetAsync(change, 0, 64, s)) return ENMF_ECUDA;
  GenArgs g;
  g.Us = U;
  g.Vs = V;
  g.W1 = W1;
  g.W2 = W2;
  g.W3 = W3;
  g.M = M;
  g.N = N;
  g.P = P;
  g.R1 = R1;
  g.R2 = R2;
  g.lam = lam;
  g.m = m;
  g.n = n;
  g.k = k;
  g.rho = rho;
  g.gamma = rho;
  g.t = rho;
  g.part = part;
  g.done = flags;
  const int stride = k * k + 4 * RMAX;
  const double thr = tol * sqrt((double)k);
  // Every step is enqueued; once the stopping rule holds (on the device,
  // after some step) the rest return at once, so the steps taken are the
  // rule's.  The host looks at the flag every check_every steps to stop
  // enqueueing.
  const int check_every = 16;
  int hflags[2] = {0, 0};
  double ch = 0.0;
  for (int it = 0; it < max_iter; ++it) {
    if (fdt == T_F64) pass<double>(0, g, s);
    else pass<float>(0, g, s);
    note_launch(1);
    gen_reduce<<<(k * k + 255) / 256, 256, 0, s>>>(part, stride, 0, k * k, Bm, flags);
    launch_polar_plain(Bm, k, R1n, D1, err, s);
    // W2 uses R2 and Lambda of the step before (Algorithm 4's f2 is separable
    // in W2 and R1) with the new W1 and W3
    if (fdt == T_F64) pass<double>(1, g, s);
    else pass<float>(1, g, s);
    note_launch(2);
    gen_reduce<<<(k * k + 255) / 256, 256, 0, s>>>(part, stride, 0, k * k, Bm, flags);
    gen_reduce<<<1, 256, 0, s>>>(part, stride, k * k, 4 * RMAX, sums, flags);
    launch_polar_plain(Bm, k, R2n, D2, err, s);
    note_launch(1);
    gen_lambda_kernel<<<1, RMAX, 0, s>>>(sums, k, lam, R1, R1n, R2, R2n, change, flags,
                                         flags + 1, thr);
    if (fdt == T_F64) pass<double>(2, g, s);
    else pass<float>(2, g, s);
    if ((it + 1) % check_every == 0) {
      if (cudaGetLastError() != cudaSuccess) return ENMF_ECUDA;
      if (cudaMemcpyAsync(hflags, flags, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        return ENMF_ECUDA;
      if (hflags[0]) break;
    }
  }
  if (cudaMemcpyAsync(&ch, change, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(hflags, flags, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(R1_out, R1, (size_t)k * k * 8, cudaMemcpyDeviceToDevice, s) ||
      cudaMemcpyAsync(R2_out, R2, (size_t)k * k * 8, cudaMemcpyDeviceToDevice, s) ||
      cudaMemcpyAsync(lam_out, lam, (size_t)k * 8, cudaMemcpyDeviceToDevice, s))
    return ENMF_ECUDA;
  // U <- U R1 Lambda R2, V <- V R1 Lambda^-1 R2
  const int bu = (int)min((int64_t)1024, (m + GR_T - 1) / GR_T);
  const int bv = (int)min((int64_t)1024, (n + GR_T - 1) / GR_T);
  note_launch(2);
  if (fdt == T_F64) {
    gen_apply<double><<<bu, GR_T, 0, s>>>((double*)U, m, k, R1, lam, R2, 0);
    gen_apply<double><<<bv, GR_T, 0, s>>>((double*)V, n, k, R1, lam, R2, 1);
  } else {
    gen_apply<float><<<bu, GR_T, 0, s>>>((float*)U, m, k, R1, lam, R2, 0);
    gen_apply<float><<<bv, GR_T, 0, s>>>((float*)V, n, k, R1, lam, R2, 1);
  }
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return ENMF_ECUDA;
  *steps_out = hflags[1];
  *change_out = ch;
  *converged = hflags[0] != 0;
  return ENMF_OK;
}

}  // namespace enmf
