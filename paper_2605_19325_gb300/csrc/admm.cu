// The ADMM rotation of Algorithm 1 for the forms with FP32 factors, every
// step of the loop inside one persistent cooperative kernel:
//   rows (all blocks)  for each row w of W = [U; V]: p = w R;
//                      y <- y + rho (z - p) from the second step on;
//                      b = p - y / rho;  z = prox(b) (Eq. 7);
//                      the block's share of M = W^T (z + y / rho);
//   M    (all blocks)  FP64 block partials, grid barrier, fixed-order sum;
//   R    (block 0)     R = polar(M), the orthogonal Procrustes solution
//                      (Sec. 4.1.2), by Newton-Schulz X <- X (3 I - X^T X) / 2
//                      in FP32 from M / ||M||_F until ||X^T X - I||_F^2 < 1e-10
//                      and one step more, then one step with X^T X in FP64:
//                      E = X^T X - I is of the order of FP32 rounding, so
//                      R = X - X E / 2 needs X E only in FP32;
//   stop               ||R_new - R||_F <= tol sqrt(r), or max_iter steps.
// Rows use eight lanes per row with the entries in registers (lanes.cuh);
// nothing returns to the host between steps.
#include "internal.h"
#include "lanes.cuh"

namespace enmf {
namespace {

using namespace lanes;

constexpr int AT = 256;          // threads per block
constexpr int ARPB = AT / LPR;   // rows per block per pass

// Dynamic shared memory (floats): Rs KP^2 | ws, bs 32 KP each | X, Y, P KP^2 each.
template <int KP>
constexpr size_t admm_smem() {
  return sizeof(float) * (4 * (size_t)KP * KP + 2 * (size_t)ARPB * KP);
}

// R = polar(M) on one block of AT threads (see the file comment).  X, Y, P:
// KP x KP shared buffers.  Thread (bi, bj) = (t / 16, t % 16) owns the
// S x S sub-block of every product.
template <int KP>
__device__ void polar_block(const double* __restrict__ Mg, int k, double* R, double tol,
                            DevState* st, int* err, float* X, float* Y, float* P, double* sh) {
  constexpr int S = KP / 16;
  const int t = threadIdx.x, bi = t / 16, bj = t % 16;
  double nf = 0.0;
  for (int e = t; e < k * k; e += AT) {
    const double v = __ldcg(&Mg[e]);
    nf = fma(v, v, nf);
  }
  nf = sqrt(block_sum256(nf, sh));
  const double inv = nf > 0.0 ? 1.0 / nf : 0.0;
  for (int e = t; e < KP * KP; e += AT) {
    const int i = e / KP, j = e % KP;
    X[e] = (i < k && j < k) ? (float)(__ldcg(&Mg[i * k + j]) * inv) : 0.f;
  }
  __syncthreads();
  int it = 0;
  for (; it < 100; ++it) {
    // P = X^T X and ||P - I||^2 over the k x k block
    float acc[S][S];
#pragma unroll
    for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) acc[s1][s2] = 0.f;
#pragma unroll
    for (int l = 0; l < KP; ++l) {
      float xa[S], xb[S];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        xa[s] = X[l * KP + bi * S + s];
        xb[s] = X[l * KP + bj * S + s];
      }
#pragma unroll
      for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2) acc[s1][s2] = fmaf(xa[s1], xb[s2], acc[s1][s2]);
    }
    float dl = 0.f;
#pragma unroll
    for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) {
        const int i = bi * S + s1, j = bj * S + s2;
        P[i * KP + j] = acc[s1][s2];
        if (i < k && j < k) {
          const float x = acc[s1][s2] - (i == j ? 1.f : 0.f);
          dl = fmaf(x, x, dl);
        }
      }
    const double dd = block_sum256((double)dl, sh);   // also orders P before its use
    // Y = 1.5 X - 0.5 X P
#pragma unroll
    for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) acc[s1][s2] = 0.f;
#pragma unroll
    for (int l = 0; l < KP; ++l) {
      float xr[S], pc[S];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        xr[s] = X[(bi * S + s) * KP + l];
        pc[s] = P[l * KP + bj * S + s];
      }
#pragma unroll
      for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2) acc[s1][s2] = fmaf(xr[s1], pc[s2], acc[s1][s2]);
    }
#pragma unroll
    for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) {
        const int e = (bi * S + s1) * KP + bj * S + s2;
        Y[e] = 1.5f * X[e] - 0.5f * acc[s1][s2];
      }
    __syncthreads();
    float* tmp = X;
    X = Y;
    Y = tmp;
    if (dd < 1e-10) {
      ++it;
      break;
    }
  }
  // E = X^T X - I with FP64 sums of the exact products (symmetric: the
  // sub-blocks with bi <= bj, mirrored), stored in FP32 in P
  if (bi <= bj) {
    double acc[S][S];
#pragma unroll
    for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) acc[s1][s2] = 0.0;
#pragma unroll
    for (int l = 0; l < KP; ++l) {
      double xa[S], xb[S];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        xa[s] = (double)X[l * KP + bi * S + s];
        xb[s] = (double)X[l * KP + bj * S + s];
      }
#pragma unroll
      for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2) acc[s1][s2] = fma(xa[s1], xb[s2], acc[s1][s2]);
    }
#pragma unroll
    for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) {
        const int i = bi * S + s1, j = bj * S + s2;
        const float e = (float)(acc[s1][s2] - (i == j && i < k ? 1.0 : 0.0));
        P[i * KP + j] = e;
        P[j * KP + i] = e;
      }
  }
  __syncthreads();
  // R_new = X - X E / 2, ||R_new - R||^2
  float acc[S][S];
#pragma unroll
  for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
    for (int s2 = 0; s2 < S; ++s2) acc[s1][s2] = 0.f;
#pragma unroll
  for (int l = 0; l < KP; ++l) {
    float xr[S], pc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      xr[s] = X[(bi * S + s) * KP + l];
      pc[s] = P[l * KP + bj * S + s];
    }
#pragma unroll
    for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) acc[s1][s2] = fmaf(xr[s1], pc[s2], acc[s1][s2]);
  }
  double d2 = 0.0;
#pragma unroll
  for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
    for (int s2 = 0; s2 < S; ++s2) {
      const int i = bi * S + s1, j = bj * S + s2;
      if (i < k && j < k) {
        const double rn = (double)X[i * KP + j] - 0.5 * (double)acc[s1][s2];
        const double x = rn - R[i * k + j];
        d2 = fma(x, x, d2);
        R[i * k + j] = rn;
      }
    }
  d2 = block_sum256(d2, sh);
  if (t == 0) {
    const double dR = sqrt(d2);
    st->dR = dR;
    st->admm_steps += 1;
    st->jac_sweeps = it;
    if (!(nf > 0.0) || it >= 100) atomicOr(err, ERR_NOTCONV);
    if (dR <= tol * sqrt((double)k)) st->admm_done = 1;
  }
}

struct AdmmArgs {
  const float* U;
  const float* V;
  int64_t m, n;
  int k;
  double* R;       // k x k FP64, R_k in, R at exit out
  float* Z;        // (m + n) x k
  float* Y;        // (m + n) x k, zero at entry
  double rho;
  int max_iter;
  double tol;
  DevState* st;
  double* part;    // grid x k x k FP64
  double* M;       // k x k FP64
  int* err;
};

template <int KP>
__global__ void __launch_bounds__(AT) admm_kernel(AdmmArgs a) {
  constexpr int E = KP / LPR, S = KP / 16;
  extern __shared__ __align__(16) unsigned char smraw[];
  float* Rs = reinterpret_cast<float*>(smraw);
  float* ws = Rs + KP * KP;
  float* bs = ws + ARPB * KP;
  float* X = bs + ARPB * KP;
  float* Yp = X + KP * KP;
  float* P = Yp + KP * KP;
  __shared__ double sh[AT];

  const int k = a.k, kk = k * k;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int sub = lane & (LPR - 1);
  const int rloc = warp * (32 / LPR) + lane / LPR;
  DevState* st = a.st;
  const int64_t m = a.m, rows = a.m + a.n;
  const int64_t passes = (rows + (int64_t)gridDim.x * ARPB - 1) / ((int64_t)gridDim.x * ARPB);
  const float rho = (float)a.rho;
  const float thr = -1.f / rho;

  for (int step = 0; step < a.max_iter; ++step) {
    if (*(volatile int*)&st->admm_done) break;   // same value in every block
    for (int e = t; e < KP * KP; e += AT) {
      const int i = e / KP, j = e % KP;
      Rs[e] = (i < k && j < k) ? (float)__ldcg(&a.R[i * k + j]) : 0.f;
    }
    __syncthreads();
    float acc[S][S];
#pragma unroll
    for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) acc[s1][s2] = 0.f;
    for (int64_t ps = 0; ps < passes; ++ps) {
      const int64_t i = (ps * gridDim.x + blockIdx.x) * ARPB + rloc;
      const bool live = i < rows;
      float w[E], z[E], y[E], p[E], bv[E];
      if (i < m) load_row(a.U, i, live, k, sub, w);
      else load_row(a.V, i - m, live, k, sub, w);
      load_row(a.Z, i, live, k, sub, z);
      load_row(a.Y, i, live, k, sub, y);
      row_times<float, KP>(Rs, w, k, sub, p);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        float yy = y[e];
        if (step > 0) yy = yy + rho * (z[e] - p[e]);   // Y update of Algorithm 1
        const float b = p[e] - yy / rho;                // b = W R - Y / rho
        const float zz = b > 0.f ? b : (b >= thr ? 0.f : b + 1.f / rho);   // Eq. 7
        z[e] = zz;
        y[e] = yy;
        bv[e] = zz + yy / rho;                          // B = Z + Y / rho
      }
      store_row(a.Z, i, live, k, sub, z);
      store_row(a.Y, i, live, k, sub, y);
      __syncthreads();
#pragma unroll
      for (int e = 0; e < E; ++e) {
        ws[rloc * KP + sub + LPR * e] = w[e];
        bs[rloc * KP + sub + LPR * e] = bv[e];
      }
      __syncthreads();
      accumulate_outer<float, KP>(ws, bs, ARPB, acc);
    }
    {
      const int bi = t / 16, bj = t % 16;
#pragma unroll
      for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
        for (int s2 = 0; s2 < S; ++s2) {
          const int pr = bi * S + s1, pc = bj * S + s2;
          if (pr < k && pc < k) a.part[(int64_t)blockIdx.x * kk + pr * k + pc] = (double)acc[s1][s2];
        }
    }
    grid_sync(&st->bar, a.err);
    sum_block_partials<AT>(a.part, (int)gridDim.x, kk, a.M);
    grid_sync(&st->bar, a.err);
    if (blockIdx.x == 0) polar_block<KP>(a.M, k, a.R, a.tol, st, a.err, X, Yp, P, sh);
    grid_sync(&st->bar, a.err);
  }
}

template <int KP>
int admm_capacity(int num_sms) {
  const size_t smem = admm_smem<KP>();
  cudaFuncSetAttribute(admm_kernel<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, admm_kernel<KP>, AT, smem);
  return (per < 1 ? 1 : per) * num_sms;
}

template <int KP>
void admm_launch(const AdmmArgs& a, int num_sms, cudaStream_t s) {
  const int64_t need = (a.m + a.n + ARPB - 1) / ARPB;
  int64_t grid = admm_capacity<KP>(num_sms);
  if (grid > NPART) grid = NPART;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  void* args[] = {(void*)&a};
  cudaLaunchCooperativeKernel((void*)admm_kernel<KP>, dim3((unsigned)grid), dim3(AT), args,
                              admm_smem<KP>(), s);
}

}  // namespace

void launch_admm_f32(const float* U, const float* V, int64_t m, int64_t n, int k, double* R,
                     float* Z, float* Y, double rho, int max_iter, double tol, DevState* st,
                     double* part, double* M, int* err, int num_sms, cudaStream_t s) {
  note_launch(1);
  AdmmArgs a{U, V, m, n, k, R, Z, Y, rho, max_iter, tol, st, part, M, err};
  const int kp = rank_pad16(k);
  if (kp == 16) admm_launch<16>(a, num_sms, s);
  else if (kp == 32) admm_launch<32>(a, num_sms, s);
  else if (kp == 48) admm_launch<48>(a, num_sms, s);
  else admm_launch<64>(a, num_sms, s);
}

}  // namespace enmf
