// The ADMM rotation of Algorithm 1 for the forms with FP32 factors, every
// step of the loop inside one persistent cooperative kernel:
//   rows (all blocks)  for each row w of W = [U; V]: p = w R;
//                      y <- y + rho (z - p) from the second step on;
//                      b = p - y / rho;  z = prox(b) (Eq. 7);
//                      the block's share of M = W^T (z + y / rho);
//   M    (all blocks)  FP64 block partials, grid barrier, fixed-order sum;
//   R    (block 0)     R = polar(M), the orthogonal Procrustes solution
//                      (Sec. 4.1.2), by scaled Newton-Schulz in FP32 from
//                      M / ||M||_F until ||X^T X - I||_F^2 < 1e-10 and one
//                      unscaled step more, then one step with X^T X - I summed
//                      in double-FP32: E is of the order of FP32 rounding, so
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

// Dynamic shared memory (floats): Rs KP^2 | ws, bs 32 KP each | X, X^T, P
// KP x PLD each (rows padded by 4 floats: 16-byte aligned, and the rows that
// eight consecutive lanes read as float4 fall in distinct banks).
template <int KP>
constexpr int polar_ld() { return KP + 4; }

template <int KP>
constexpr size_t admm_smem() {
  return sizeof(float) * ((size_t)KP * KP + 2 * (size_t)ARPB * KP + 3 * (size_t)KP * polar_ld<KP>());
}

// acc[s1][s2] += sum_l A[ia_s1][l] B[jb_s2][l] over l < KP, with rows
// ia_s = bi + 16 s of A and jb_s = bj + 16 s of B (row stride LD), read as
// float4 along l.
template <int KP, int LD>
__device__ __forceinline__ void rows_dot(const float* __restrict__ A, const float* __restrict__ Bm,
                                         int bi, int bj, float (&acc)[KP / 16][KP / 16]) {
  constexpr int S = KP / 16;
#pragma unroll
  for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
    for (int s2 = 0; s2 < S; ++s2) acc[s1][s2] = 0.f;
#pragma unroll 4
  for (int l = 0; l < KP; l += 4) {
    float4 x[S], y[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      x[s] = *reinterpret_cast<const float4*>(A + (bi + 16 * s) * LD + l);
      y[s] = *reinterpret_cast<const float4*>(Bm + (bj + 16 * s) * LD + l);
    }
#pragma unroll
    for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) {
        float c = acc[s1][s2];
        c = fmaf(x[s1].x, y[s2].x, c);
        c = fmaf(x[s1].y, y[s2].y, c);
        c = fmaf(x[s1].z, y[s2].z, c);
        c = fmaf(x[s1].w, y[s2].w, c);
        acc[s1][s2] = c;
      }
  }
}

// Power iteration on I - P (P = X_0^T X_0, symmetric, eigenvalues in [0, 1])
// by warp 0, from the vector v of the previous call: the Rayleigh quotient mu
// gives sigma_min(X_0)^2 ~ 1 - mu (from above).  v: KP floats, zero past k.
template <int KP, int LD>
__device__ float sigma_min_estimate(const float* __restrict__ P, float* v, int k, int iters) {
  constexpr int E = (KP + 31) / 32;
  const int lane = threadIdx.x & 31;
  float w[E], mu = 0.f;
  for (int t = 0; t <= iters; ++t) {
#pragma unroll
    for (int e = 0; e < E; ++e) w[e] = lane + 32 * e < KP ? v[lane + 32 * e] : 0.f;
    for (int j = 0; j < k; ++j) {
      const float vj = v[j];
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (lane + 32 * e < KP) w[e] = fmaf(-P[j * LD + lane + 32 * e], vj, w[e]);
    }
    float nn = 0.f, vw = 0.f;
#pragma unroll
    for (int e = 0; e < E; ++e)
      if (lane + 32 * e < KP) {
        nn = fmaf(w[e], w[e], nn);
        vw = fmaf(v[lane + 32 * e], w[e], vw);
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      nn += __shfl_xor_sync(FULL, nn, o);
      vw += __shfl_xor_sync(FULL, vw, o);
    }
    mu = vw;                                  // v is a unit vector
    if (t == iters || !(nn > 0.f)) break;
    const float inv = rsqrtf(nn);
    __syncwarp();
#pragma unroll
    for (int e = 0; e < E; ++e)
      if (lane + 32 * e < KP) v[lane + 32 * e] = w[e] * inv;
    __syncwarp();
  }
  return sqrtf(fmaxf(1.f - mu, 0.f));
}

// R = polar(M) on one block of AT threads (see the file comment).  X, XT, P:
// KP x PLD shared buffers; v: KP floats kept from step to step.  Thread
// (bi, bj) = (t / 16, t % 16) owns the entries (bi + 16 s1, bj + 16 s2).
//
// The iteration is Newton-Schulz with the scaling of a lower bound l of the
// singular values (X <- alpha X (3 I - alpha^2 X^T X) / 2, alpha^2 =
// 3 / (1 + l + l^2), which maps [l, 1] into [l', 1] with l' = alpha l (3 -
// alpha^2 l^2) / 2): for every singular value in (0, 1] it stays in (0, 1]
// and grows at least as fast as the unscaled step, so the limit is the same
// polar factor whatever l is; l only sets the speed.  l starts from a power
// iteration on I - X_0^T X_0 and is raised to sqrt(1 - ||X^T X - I||_F) once
// that bound holds; the step after convergence is unscaled.
template <int KP>
__device__ void polar_block(const double* __restrict__ Mg, int k, double* R, double tol,
                            DevState* st, int* err, float* X, float* XT, float* P, float* v,
                            bool first, double* sh) {
  constexpr int S = KP / 16, LD = polar_ld<KP>();
  const int t = threadIdx.x, bi = t / 16, bj = t % 16;
  double nf = 0.0;
  for (int e = t; e < k * k; e += AT) {
    const double x = __ldcg(&Mg[e]);
    nf = fma(x, x, nf);
  }
  nf = sqrt(block_sum256(nf, sh));
  const double inv = nf > 0.0 ? 1.0 / nf : 0.0;
  for (int e = t; e < KP * KP; e += AT) {
    const int i = e / KP, j = e % KP;
    const float x = (i < k && j < k) ? (float)(__ldcg(&Mg[i * k + j]) * inv) : 0.f;
    X[i * LD + j] = x;
    XT[j * LD + i] = x;
  }
  if (first)
    for (int i = t; i < KP; i += AT) v[i] = i < k ? 1.f + 0.25f * (float)(i % 5) : 0.f;
  __syncthreads();
  float* lsh = reinterpret_cast<float*>(sh) + 8;   // past block_sum256f's 8 floats
  float lk = 0.f;
  int it = 0;
  for (; it < 100; ++it) {
    float acc[S][S], xo[S][S];
    rows_dot<KP, LD>(XT, XT, bi, bj, acc);      // P = X^T X
    float dl = 0.f;
#pragma unroll
    for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) {
        const int i = bi + 16 * s1, j = bj + 16 * s2;
        P[i * LD + j] = acc[s1][s2];
        xo[s1][s2] = X[i * LD + j];
        if (i < k && j < k) {
          const float x = acc[s1][s2] - (i == j ? 1.f : 0.f);
          dl = fmaf(x, x, dl);
        }
      }
    // ||P - I||_F^2 in FP32 (its threshold 1e-10 is far above FP32 rounding);
    // the barriers inside also order P before its use
    const float dd = block_sum256f(dl, reinterpret_cast<float*>(sh));
    if (it == 0) {
      if (t < 32) {
        float l0 = sigma_min_estimate<KP, LD>(P, v, k, first ? 12 : 3);
        if (t == 0) lsh[0] = fminf(fmaxf(0.9f * l0, 1e-4f), 1.f);
      }
      __syncthreads();
      lk = lsh[0];
    }
    const bool conv = dd < 1e-10f;
    if (dd < 1.f) lk = fmaxf(lk, sqrtf(fmaxf(1.f - sqrtf(dd), 0.f)));
    const float al = conv ? 1.f : sqrtf(3.f / (1.f + lk + lk * lk));
    const float ca = 1.5f * al, cb = 0.5f * al * al * al;
    lk = 0.5f * al * lk * (3.f - al * al * lk * lk);
    rows_dot<KP, LD>(X, P, bi, bj, acc);        // X P  (P symmetric)
    __syncthreads();                            // every read of X, X^T, P done
#pragma unroll
    for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) {
        const int i = bi + 16 * s1, j = bj + 16 * s2;
        const float y = ca * xo[s1][s2] - cb * acc[s1][s2];
        X[i * LD + j] = y;
        XT[j * LD + i] = y;
      }
    __syncthreads();
    if (conv) {
      ++it;
      break;
    }
  }
  // E = X^T X - I to about 2^-44: each product split exactly (x y = p + e by
  // one FMA) and the p summed with an exact two-sum, the errors in FP32 (the
  // sub-blocks with bi <= bj, mirrored); E itself is of the order of FP32
  // rounding, so R = X - X E / 2 needs X E only in FP32
  if (bi <= bj) {
#pragma unroll
    for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
      for (int s2 = 0; s2 < S; ++s2) {
        const int i = bi + 16 * s1, j = bj + 16 * s2;
        const float* xi = XT + i * LD;
        const float* xj = XT + j * LD;
        float hi = 0.f, lo = 0.f;
        for (int l = 0; l < KP; ++l) {
          const float p = __fmul_rn(xi[l], xj[l]);
          const float pe = fmaf(xi[l], xj[l], -p);
          const float sm = __fadd_rn(hi, p);
          const float bv = __fsub_rn(sm, hi);
          const float er = __fadd_rn(__fsub_rn(hi, __fsub_rn(sm, bv)), __fsub_rn(p, bv));
          hi = sm;
          lo = __fadd_rn(lo, __fadd_rn(er, pe));
        }
        const float e = __fadd_rn(__fsub_rn(hi, (i == j && i < k) ? 1.f : 0.f), lo);
        P[i * LD + j] = e;
        P[j * LD + i] = e;
      }
  }
  __syncthreads();
  // R_new = X - X E / 2 (E symmetric), ||R_new - R||^2
  float acc[S][S];
  rows_dot<KP, LD>(X, P, bi, bj, acc);
  double d2 = 0.0;
#pragma unroll
  for (int s1 = 0; s1 < S; ++s1)
#pragma unroll
    for (int s2 = 0; s2 < S; ++s2) {
      const int i = bi + 16 * s1, j = bj + 16 * s2;
      if (i < k && j < k) {
        const double rn = (double)X[i * LD + j] - 0.5 * (double)acc[s1][s2];
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
  float* XT = X + KP * polar_ld<KP>();
  float* P = XT + KP * polar_ld<KP>();
  __shared__ double sh[AT];
  __shared__ float pv[KP];

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
    if (blockIdx.x == 0)
      polar_block<KP>(a.M, k, a.R, a.tol, st, a.err, X, XT, P, pv, step == 0, sh);
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
